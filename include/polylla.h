/*
 * polylla.h -- C ABI of the GB300 terminal-edge-region polygonal mesher.
 *
 * Implements the GPU algorithm of Salinas, Ojeda, Hitschfeld and Ortiz-Bernardin,
 * "GPU parallel algorithm for the generation of polygonal meshes based on
 * terminal-edge regions" (IMR 2022): label every edge of a 2D triangulation
 * (Section 3.2.1, Algorithm 2), build one polygon per terminal-edge region
 * (Section 3.2.2, Algorithms 3 and 4) and split non-simple polygons at their
 * barrier-edge tips (Section 3.2.3, Algorithm 5), driven as in Algorithm 1.
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 * Mesh layout (Section 2, with an explicit half-edge twin in place of the
 * Neighbor array):
 *   xy   int64[2n]  device; xy[2v], xy[2v+1] = lattice coordinates of vertex v,
 *                   each in [0, 2^30) (exact int64 squared lengths).
 *   tri  int32[3m]  device; tri[3t+k] = k-th vertex of triangle t, ccw, with
 *                   positive area.  Half-edge h = 3t+k runs from tri[h] to
 *                   tri[3t+(k+1)%3].
 *   twin int32[3m]  device; the opposite half-edge of h, or -1 on the border.
 * Sizes: 3 <= n < 2^30, 1 <= m < 2^29 (half-edge ids fit int32; the output scan
 * packs a polygon count and a vertex count in one 64-bit word).
 *
 * Ownership: the input arrays are borrowed, never written, and must stay valid
 * until polylla_mesh_destroy.  Every derived array (labels, seeds, polygons) is
 * owned by the handle; pointers returned by the getters stay valid until the
 * next phase call on the handle or its destruction.
 *
 * Ordering: every call is asynchronous on the given stream (a cudaStream_t passed
 * as void*; NULL = the legacy default stream), except the calls documented as
 * synchronising.  One handle must not be used from two streams at once.
 *
 * Errors: every call returns a polylla_status and never throws.  Errors found on
 * the device (an index out of range, a walk or reparation exceeding its bound)
 * are recorded in a per-handle device word and reported by the next
 * synchronising call.  Phases must run in order label -> seeds -> traverse ->
 * repair (polylla_label may restart the pipeline at any time), else
 * POLYLLA_ERR_STATE.
 *
 * Label byte lab[t] (one per triangle):
 *   bits 0-1  index k (0..2) of the longest edge of t (the Max array, Section 2);
 *             lengths are exact squared lengths, ties go to the edge with the
 *             lower undirected id min(h, twin(h)) (a reading: the paper gives no
 *             tie rule);
 *   bit 2+k   edge k of t is a frontier edge (LabelFrontier, Algorithm 2);
 *   bit 5     t is a seed triangle (LabelSeed, Algorithm 2; the Seed array);
 *   bit 6     the longest edge of t is a terminal edge.
 * An edge that is neither frontier nor terminal is an internal edge.
 *
 * Polygons: CSR, int64 off[np+1] and int32 vtx[off[np]]; polygon i is
 * vtx[off[i] .. off[i+1]), ccw, starting at its frontier half-edge with the
 * smallest (origin vertex, half-edge id) -- i.e. at its smallest vertex id once
 * simple.  After traversal polygon i belongs to the i-th seed in ascending
 * order; reparation replaces each split polygon, in place, by its two halves
 * (recursively), the half containing the new half-edge tip->x first.
 */
#ifndef POLYLLA_H
#define POLYLLA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct polylla_mesh* polylla_mesh_t;

typedef enum {
  POLYLLA_OK = 0,
  POLYLLA_ERR_INVALID_ARG = 1, /* null pointer, bad size, unknown flag */
  POLYLLA_ERR_RANGE = 2,       /* coordinate outside [0, 2^30), id out of range */
  POLYLLA_ERR_TOPOLOGY = 3,    /* twin not consistent, triangle not ccw / degenerate */
  POLYLLA_ERR_OOM = 4,         /* device allocation failed */
  POLYLLA_ERR_CUDA = 5,        /* a CUDA runtime call failed */
  POLYLLA_ERR_LIMIT = 6,       /* a walk or a reparation exceeded its bound */
  POLYLLA_ERR_STATE = 7,       /* phase called out of order */
  POLYLLA_ERR_CANCELLED = 8    /* served request cancelled before it was admitted */
} polylla_status;

#define POLYLLA_VALIDATE 1u /* mesh_create checks the mesh on the device (synchronises) */

#define POLYLLA_LAB_MAX_MASK 0x03u
#define POLYLLA_LAB_FRONTIER_SHIFT 2
#define POLYLLA_LAB_SEED 0x20u
#define POLYLLA_LAB_TERMINAL 0x40u

/* Statistics of the last completed pipeline (polylla_get_stats). */
typedef struct {
  int64_t n_seeds;        /* seeds = terminal-edge regions */
  int64_t n_poly_trav;    /* polygons after traversal (= n_seeds) */
  int64_t n_vtx_trav;     /* their total length (= frontier half-edges) */
  int64_t n_tip_polygons; /* polygons with at least one barrier-edge tip */
  int64_t n_tips;         /* barrier-edge tips found by traversal */
  int64_t n_splits;       /* splits made by reparation */
  int64_t n_poly;         /* polygons after reparation */
  int64_t n_vtx;          /* their total length */
  /* Which device path handled the polygons of the last traversal / reparation
   * pass (every path gives the same polygons; these show which ones ran): */
  int64_t n_long;         /* polygons longer than the thread walk's cap (and, on
                             meshes of fewer than 2^16 triangles, polygons with three
                             or more tips), walked and split by one thread block each */
  int64_t n_long_handoff; /* of those, regions a small block could not hold and
                             handed to a large one (batch schedules with long_mode 1, 2) */
  int64_t n_long_seq;     /* of those, regions too large for any block's shared
                             memory, walked and split by one thread */
  int64_t n_one_tip;      /* polygons with exactly one tip, split by the one-tip kernel */
  int64_t n_multi_tip;    /* polygons with several tips, split in shared memory */
  int64_t n_multi_seq;    /* of those, polygons with more tips than the shared node
                             list holds, split by re-walking */
  int64_t n_one_chase;    /* one-tip polygons whose pieces could not be cut out of the
                             traversal's vertex sequence (a repeated vertex), split by
                             chasing the successors */
  int64_t n_multi_turn;   /* pieces of several-tip polygons whose smallest vertex
                             repeats, their half-edges found by turning */
  int64_t n_one_block;    /* polygons of a small mesh meshed, whole path, by one
                             thread block (polylla_run; see polylla_set_one_block) */
} polylla_stats;

/*
 * Create a handle over a device-resident triangulation (Section 2's arrays).
 * d_xy, d_tri, d_twin: device pointers as described above (borrowed).  d_twin may
 * be NULL: the handle then builds the twin array from tri on the device (its
 * Neighbor array comes from the triangulator in the paper, Section 2) and
 * synchronises; a directed edge used twice or an edge with more than two
 * triangles gives POLYLLA_ERR_TOPOLOGY.  flags: 0 or POLYLLA_VALIDATE; with
 * VALIDATE the mesh is checked on the device (ids and twins in range, twin an
 * involution between reversed edges, coordinates in range, every triangle ccw
 * with positive area) and the call synchronises with `stream`.  Allocates every
 * derived buffer (about 190 bytes per triangle) so that later phases allocate
 * nothing.  On success *out receives the handle; on failure *out is NULL.
 */
polylla_status polylla_mesh_create(const int64_t* d_xy, int64_t n_vertices, const int32_t* d_tri,
                                   int64_t n_tri, const int32_t* d_twin, uint32_t flags,
                                   void* stream, polylla_mesh_t* out);

/*
 * Create a handle from the triangulator's Neighbor array instead of a twin array
 * (Section 2: Triangle, QHull and Detri2 write it; the paper's inputs are
 * Triangle's .node / .ele / .neigh files).  d_neighbor: device int32[3m],
 * 4-byte aligned, borrowed for the call only; d_neighbor[3t + j] is the triangle
 * across edge j of triangle t, or -1 on the border.  convention
 * POLYLLA_NEIGHBOR_OPPOSITE: edge j is the edge opposite vertex tri[3t + j]
 * (Triangle's .neigh layout); POLYLLA_NEIGHBOR_EDGE: edge j is the edge from
 * tri[3t + j] to tri[3t + (j+1) % 3] (half-edge 3t + j).  The handle owns the
 * twin array it builds on the device (the twin of u -> v is the neighbour's
 * v -> u) and synchronises with `stream`; a neighbour id outside [-1, m) gives
 * POLYLLA_ERR_RANGE, a neighbour without the reversed edge POLYLLA_ERR_TOPOLOGY.
 * Otherwise as polylla_mesh_create (d_xy, d_tri 16-byte aligned; flags 0 or
 * POLYLLA_VALIDATE).
 *
 * polylla_get_twin: the device twin array the handle uses (borrowed or built),
 * valid until destroy.
 */
#define POLYLLA_NEIGHBOR_OPPOSITE 0
#define POLYLLA_NEIGHBOR_EDGE 1
polylla_status polylla_mesh_create_neighbors(const int64_t* d_xy, int64_t n_vertices,
                                             const int32_t* d_tri, int64_t n_tri,
                                             const int32_t* d_neighbor, int convention,
                                             uint32_t flags, void* stream, polylla_mesh_t* out);
polylla_status polylla_get_twin(polylla_mesh_t mesh, const int32_t** d_twin);

/*
 * The Trivertex array (Section 2: one element incident to each vertex; the
 * paper's reparation finds a tip's fan through it, Section 3.2.3): for every
 * vertex v, the smallest half-edge id leaving v (its triangle is id / 3), or -1
 * for a vertex no triangle uses.  polylla_trivertex computes it on `stream`
 * (asynchronous; any time after creation); polylla_get_trivertex (synchronises,
 * reports a vertex id out of range) returns the handle-owned device int32[n],
 * valid until the handle's triangles change or it is destroyed;
 * POLYLLA_ERR_STATE before polylla_trivertex.
 */
polylla_status polylla_trivertex(polylla_mesh_t mesh, void* stream);
polylla_status polylla_get_trivertex(polylla_mesh_t mesh, const int32_t** d_trivertex);

/*
 * Label phase (Section 3.2.1, Algorithm 2): LabelMax, then LabelSeed and
 * LabelFrontier fused in one pass, writing lab[m] (layout above).  Restarts the
 * pipeline.  Asynchronous.
 */
polylla_status polylla_label(polylla_mesh_t mesh, void* stream);

/*
 * Seeds (Section 3.2.1, the Seed array): the seed triangles compacted in
 * ascending order into a device int32 list, with its length kept on the device.
 * Asynchronous.
 */
polylla_status polylla_seeds(polylla_mesh_t mesh, void* stream);

/*
 * Traversal phase (Section 3.2.2, Algorithms 3 and 4): one polygon per seed, in
 * seed order, written as CSR (the Mesh and Position arrays) at offsets given by a
 * scan instead of the paper's atomicAdd.  Polygons may be non-simple.
 * Asynchronous.
 */
polylla_status polylla_traverse(polylla_mesh_t mesh, void* stream);

/*
 * Reparation phase (Section 3.2.3, Algorithm 5 with the loop of Algorithm 1):
 * every polygon with barrier-edge tips is split at its smallest tip vertex along
 * the middle internal edge e_ceil(k/2) (k internal edges at the tip, counted ccw
 * after the barrier edge), which becomes a frontier edge in lab[], repeatedly
 * until no tips remain.  Writes the final CSR.  Asynchronous.
 */
polylla_status polylla_repair(polylla_mesh_t mesh, void* stream);

/*
 * The reparation phase on the host: the paper's mixed variant (Section 3.2 and
 * Section 4 compare GPU labelling and traversal followed by a sequential CPU
 * reparation with the all-GPU path).  After polylla_traverse, copies the mesh, the
 * label bytes and the traversal polygons to host memory, repairs them with one
 * host thread (Section 3.2.3: each polygon's tips split in turn at the middle
 * internal edge of the tip's fan, found through the Trivertex array; the same
 * readings as polylla_repair), and copies the final polygons and label bytes
 * back.  Afterwards the getters report exactly what they report after
 * polylla_repair (the per-path counters of the device kernels stay 0).
 * Synchronises; POLYLLA_ERR_STATE unless the last phase was polylla_traverse;
 * POLYLLA_ERR_LIMIT if a polygon cannot be repaired (a corrupt mesh).
 */
polylla_status polylla_repair_host(polylla_mesh_t mesh, void* stream);

/*
 * Algorithm 1 end to end: label, seeds, traversal and reparation.  The final
 * polygons and labels equal those of the four phase calls; the pre-reparation
 * CSR is not materialised.  Asynchronous.
 *
 * A mesh of at most polylla_set_one_block's limit of triangles (default
 * polylla_one_block_limit() = 4096) is meshed by one launch of one thread block
 * that holds the whole half-edge state in shared memory: Algorithm 2's labels,
 * the Seed array, Algorithm 4's walks and Algorithm 5's splits (each polygon
 * with tips split by the thread that walked it, smallest tip first) and the CSR,
 * with the same results as the multi-kernel path (statistic n_one_block counts
 * its polygons; the other per-path counters stay 0).  Larger meshes take the
 * multi-kernel path, whose kernels each spread over the whole GPU.
 */
polylla_status polylla_run(polylla_mesh_t mesh, void* stream);

/*
 * The largest mesh (in triangles) that polylla_run gives to the one-block path,
 * 0 .. polylla_one_block_limit() (0: always the multi-kernel path).  Takes
 * effect at the next polylla_run.  POLYLLA_ERR_INVALID_ARG for a null handle or
 * a value out of range.  No device call.
 */
polylla_status polylla_set_one_block(polylla_mesh_t mesh, int64_t max_triangles);
int64_t polylla_one_block_limit(void);

/* Device pointer to lab[m] (valid after polylla_label; updated by repair). */
polylla_status polylla_get_labels(polylla_mesh_t mesh, const uint8_t** d_lab);

/* Device pointer to the seed list and its length.  Synchronises. */
polylla_status polylla_get_seeds(polylla_mesh_t mesh, const int32_t** d_seeds, int64_t* n_seeds);

/* Device pointers to the latest CSR (after traverse: pre-reparation; after
 * repair or run: final) and its sizes.  Synchronises. */
polylla_status polylla_get_polygons(polylla_mesh_t mesh, const int64_t** d_off,
                                    const int32_t** d_vtx, int64_t* n_poly, int64_t* n_vtx);

/* Statistics of the pipeline so far (fields of later phases are 0).  Synchronises. */
polylla_status polylla_get_stats(polylla_mesh_t mesh, polylla_stats* out);

/* Release every buffer of the handle (synchronises with the device). */
polylla_status polylla_mesh_destroy(polylla_mesh_t mesh);

/* Static, human-readable name of a status. */
const char* polylla_status_str(polylla_status status);

/*
 * End-to-end call from HOST memory: copies xy, tri, twin from host buffers
 * (pinned memory recommended) into device buffers owned by `mesh`, runs
 * polylla_run, and copies the final CSR back into host buffers.  `mesh` must
 * have been created with polylla_mesh_create_host.  h_twin may be NULL: the twin
 * array is then built on the device from tri (one copy less).  h_off needs room
 * for n_tri+1 entries and h_vtx for 3*n_tri (the bounds of the final mesh).
 * Synchronises.
 *
 * polylla_mesh_build_twin: for a handle that owns its twin array (created with
 * d_twin NULL, or by polylla_mesh_create_host), rebuilds it from the current tri
 * on the device; asynchronous (errors at the next synchronising call); the
 * phases restart.
 */
polylla_status polylla_mesh_create_host(int64_t n_vertices, int64_t n_tri, polylla_mesh_t* out);
polylla_status polylla_run_host(polylla_mesh_t mesh, const int64_t* h_xy, const int32_t* h_tri,
                                const int32_t* h_twin, int64_t* h_off, int32_t* h_vtx,
                                int64_t* n_poly, int64_t* n_vtx, void* stream);
polylla_status polylla_mesh_build_twin(polylla_mesh_t mesh, void* stream);

/*
 * Per-kernel timing: when enabled, every kernel the handle launches is bracketed
 * by CUDA events on its stream.  polylla_kernel_times fills up to `cap` entries
 * (name, milliseconds) of the launches since the last reset, synchronising, and
 * returns the number of launches recorded.  polylla_launch_count returns the
 * number of kernels launched by the handle since creation.
 */
polylla_status polylla_set_timing(polylla_mesh_t mesh, int enable);
int64_t polylla_kernel_times(polylla_mesh_t mesh, const char** names, float* ms, int64_t cap,
                             int reset);
int64_t polylla_launch_count(polylla_mesh_t mesh);

/*
 * Allocation-free label phase and seed compaction.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory (a host
 * that owns the whole device heap, or code that must not let cudaMalloc /
 * cudaFree synchronise the device).  It computes exactly what polylla_label
 * followed by polylla_seeds computes, without a handle, and allocates nothing:
 * its only scratch (the seed compaction's look-back words, counters and an error
 * word) lives in a fixed file-scope device array of about 33 KiB, which every GPU
 * that loads the library holds until the process exits.
 *   d_xy, n_vertices, d_tri, d_twin, n_tri: the mesh, as for polylla_mesh_create
 *     (16-byte aligned), with at most 2^26 triangles -- larger meshes are rejected
 *     with POLYLLA_ERR_INVALID_ARG;
 *   d_lab: device uint8[n_tri], 4-byte aligned, receives the label bytes;
 *   d_seeds: device int32[n_tri] (capacity), receives the ascending seed list;
 *   d_n_seeds: one device int64, 8-byte aligned, receives the seed count.
 * The array and the entry point's kernels are loaded onto a device by the first
 * call on that device (the CUDA runtime loads device code lazily): that first call
 * allocates their device memory and may synchronise the device.  A caller that
 * reserves all device memory for its own arena therefore makes one call (on any
 * small mesh) per device before reserving it; later calls allocate nothing.  The array's address is looked up on every call
 * with the calling device current.  Every call shares the one array and clears
 * what must start at zero, so calls that overlap on the GPU race and must be
 * serialised by the caller.  Each call waits for `stream` to finish before
 * returning, to report device-side errors.
 */
polylla_status polylla_label_seeds_noalloc(const int64_t* d_xy, int64_t n_vertices,
                                           const int32_t* d_tri, const int32_t* d_twin,
                                           int64_t n_tri, uint8_t* d_lab, int32_t* d_seeds,
                                           int64_t* d_n_seeds, void* stream);

/*
 * Longest-edge propagation paths (Section 2's Lepp, which defines terminal-edge
 * regions; Lepp-based kernels are the paper's future work, Section 5), from the
 * label phase's Max array.  For every triangle t, following the neighbour across
 * the longest edge until that edge is terminal (the longest edge of both its
 * triangles, or a border edge): region[t] is the seed of the terminal edge reached
 * (its lower triangle, or the border triangle) -- the seed of t's terminal-edge
 * region -- and depth[t] the number of links followed.
 * polylla_lepp: after polylla_label (any later phase keeps the Max array);
 * asynchronous.  polylla_get_lepp (synchronises, reports a path error): device
 * int32[m] arrays owned by the handle, valid until the next polylla_label or
 * destroy; POLYLLA_ERR_STATE before polylla_lepp.
 */
polylla_status polylla_lepp(polylla_mesh_t mesh, void* stream);
polylla_status polylla_get_lepp(polylla_mesh_t mesh, const int32_t** d_region,
                                const int32_t** d_depth);

/*
 * Batches: many independent meshes in one run (the paper meshes one
 * triangulation at a time; this form has no counterpart there).
 *
 * The meshes are given concatenated, with mesh-local ids:
 *   d_xy      int64[2 * vtx_off[n]]: mesh j's vertices are rows vtx_off[j] ..
 *             vtx_off[j+1]-1 (16-byte aligned; borrowed until destroy);
 *   d_tri     int32[3 * tri_off[n]]: mesh j's triangles are tri_off[j] ..
 *             tri_off[j+1]-1, their vertex ids local to mesh j (0-based);
 *   d_twin    int32[3 * tri_off[n]]: twins as half-edge ids local to mesh j, or -1;
 *   d_vtx_off, d_tri_off  device int64[n_meshes + 1], starting at 0, each mesh
 *             with >= 3 vertices and >= 1 triangle; totals as for one mesh
 *             (< 2^30 vertices, < 2^29 triangles).
 * polylla_batch_create copies the offsets to the host (synchronises), rewrites
 * the ids into one disjoint union mesh on the device (handle-owned; local ids
 * out of range give POLYLLA_ERR_RANGE) and, with POLYLLA_VALIDATE, checks it as
 * polylla_mesh_create does.
 *
 * polylla_batch_run runs the whole path (label, seeds, traversal, reparation) on
 * every mesh at once: the union is meshed exactly as one mesh would be, so each
 * mesh's polygons are exactly those it gives alone.  The launches of a schedule
 * are captured into a CUDA graph on its first use (that call runs eagerly) and
 * replayed afterwards.  schedule: 0 .. polylla_batch_schedules()-1, or
 * POLYLLA_SCHEDULE_TUNED for the one polylla_batch_tune picked (tuning first if
 * needed).  A schedule sets the longest polygon walked by one thread (longer
 * ones go to one thread block each) and how those blocks are sized (long_mode 0:
 * one large block per polygon; 1: small blocks first, several per SM, handing
 * the regions they cannot hold to large ones; 2: the same with one warp per
 * polygon first) and whether the three kernels after
 * the walk overlap on side streams (overlap 1) or run one after another (0);
 * polylla_batch_schedule_info reports all three.
 *
 * polylla_batch_tune times every schedule on this batch (`reps` graph replays
 * each, after one warm-up), stores the fastest, and returns it in *best and the
 * mean milliseconds per run in ms[k] (either may be NULL).  Synchronises.
 *
 * polylla_batch_get (synchronises): mesh j's polygons.  *d_off points at
 * n_poly + 1 offsets into *d_vtx (the whole batch's vertex array); polygon k's
 * vertices are (*d_vtx)[(*d_off)[k] .. (*d_off)[k+1]).  Vertex ids index the
 * concatenated d_xy (subtract vtx_off[j] for mesh-local ids).  n_vtx is the
 * mesh's vertex-slot count.  polylla_batch_get_all returns the whole CSR and
 * d_mesh_first (n_meshes + 1 polygon indices: mesh j owns polygons
 * d_mesh_first[j] .. d_mesh_first[j+1]-1).  The pointers stay valid until the
 * next run or destroy.  polylla_batch_mesh returns the union's handle (for
 * statistics and timing; do not destroy it).
 */
typedef struct polylla_batch* polylla_batch_t;
#define POLYLLA_SCHEDULE_TUNED (-1)

polylla_status polylla_batch_create(const int64_t* d_xy, const int64_t* d_vtx_off,
                                    const int32_t* d_tri, const int32_t* d_twin,
                                    const int64_t* d_tri_off, int64_t n_meshes, uint32_t flags,
                                    void* stream, polylla_batch_t* out);
int polylla_batch_schedules(void);
polylla_status polylla_batch_schedule_info(int schedule, int* walk_cap, int* long_mode,
                                           int* overlap);
polylla_status polylla_batch_tune(polylla_batch_t batch, int reps, void* stream, int* best,
                                  float* ms);
polylla_status polylla_batch_run(polylla_batch_t batch, int schedule, void* stream);
polylla_status polylla_batch_get(polylla_batch_t batch, int64_t mesh, const int64_t** d_off,
                                 const int32_t** d_vtx, int64_t* n_poly, int64_t* n_vtx);
polylla_status polylla_batch_get_all(polylla_batch_t batch, const int64_t** d_off,
                                     const int32_t** d_vtx, const int64_t** d_mesh_first,
                                     int64_t* n_poly, int64_t* n_vtx);
polylla_status polylla_batch_stats(polylla_batch_t batch, polylla_stats* out);
polylla_mesh_t polylla_batch_mesh(polylla_batch_t batch);
polylla_status polylla_batch_destroy(polylla_batch_t batch);

/*
 * Capacity handles and asynchronous results (for callers that reuse device
 * state across meshes, such as the server below).
 *
 * polylla_mesh_footprint: device bytes a handle for n vertices and m triangles
 * allocates (owns_inputs != 0: also its input arrays, as polylla_mesh_create_host
 * does); -1 for invalid sizes.  No device call.
 * polylla_mesh_set_size: for a handle created by polylla_mesh_create_host, the
 * size of the next mesh (at most its creation sizes); the phases restart.
 * polylla_mesh_inputs: the device input arrays of such a handle, to fill
 * (asynchronously) before polylla_run.
 * polylla_get_polygons_async: like polylla_get_polygons without synchronising:
 * the latest CSR's device pointers, plus d_counts (int64[2]: n_poly, n_vtx) and
 * d_error (the handle's int32 device error word, 0 if none), valid on the
 * handle's stream once the phase that wrote them has run.
 */
int64_t polylla_mesh_footprint(int64_t n_vertices, int64_t n_tri, int owns_inputs);
polylla_status polylla_mesh_set_size(polylla_mesh_t mesh, int64_t n_vertices, int64_t n_tri);
polylla_status polylla_mesh_inputs(polylla_mesh_t mesh, int64_t** d_xy, int32_t** d_tri,
                                   int32_t** d_twin);
polylla_status polylla_get_polygons_async(polylla_mesh_t mesh, const int64_t** d_off,
                                          const int32_t** d_vtx, const int64_t** d_counts,
                                          const int32_t** d_error);

/*
 * Served form: a request loop with continuous batching (no counterpart in the
 * paper).  polylla_server_create starts a worker thread and a slot-creating
 * thread on the current device with a device-memory budget (bytes, >= 1 MiB) and
 * at most max_slots resident slots.  A slot is a capacity handle for a size class (the smallest power of two
 * c >= max(4096, m, 2n) triangles, up to c/2 + 2 vertices) whose device state
 * stays allocated and serves the next request of its class, or of a smaller
 * class (up to 8x smaller) when no slot of that class is free.
 *
 * polylla_server_submit queues one mesh (host arrays as for polylla_run_host;
 * pinned memory lets the copies overlap; h_twin NULL: built on the device) and
 * returns its id.  h_off_out
 * (int64[m+1]) and h_vtx_out (int32[3m]) receive the final CSR.  Every buffer
 * must stay valid until the request completes.  Requests are admitted in arrival
 * order as soon as a slot of their class is free; otherwise, when a new slot fits
 * the budget (idle slots of other classes are released to make room), it is
 * allocated by the slot-creating thread while the requests on the device go on,
 * and the request waits for it.  When a request takes the last idle slot that can
 * serve its class, a spare of that class is allocated the same way if it fits
 * the budget and leaves one slot of max_slots free.  A request whose class alone
 * exceeds the budget, or whose slot cannot be allocated, completes with
 * POLYLLA_ERR_OOM.  Admitted requests run on their slots' streams and overlap on
 * the device; each is meshed by its own handle, so its result is the same as
 * alone.  bytes_in_use (polylla_server_info) counts the slots being allocated.
 *
 * polylla_server_poll moves up to `cap` completed results into out[], waiting up
 * to wait_us microseconds for the first, and returns how many (-1 on bad
 * arguments).  Times are seconds since the server's creation.
 * polylla_server_info reports its state; polylla_server_destroy finishes every
 * queued and running request, then frees everything.
 */
typedef struct polylla_server* polylla_server_t;
typedef struct {
  int64_t id;
  int32_t status;   /* POLYLLA_OK, or the request's error */
  int32_t reserved;
  int64_t n_poly, n_vtx;
  double submit_s, admit_s, done_s;
} polylla_result;
typedef struct {
  int64_t slots, bytes_in_use, budget_bytes, pending, running, peak_running, completed;
  double now_s;
} polylla_server_stats;

polylla_status polylla_server_create(int64_t budget_bytes, int max_slots, polylla_server_t* out);
polylla_status polylla_server_submit(polylla_server_t server, const int64_t* h_xy,
                                     int64_t n_vertices, const int32_t* h_tri,
                                     const int32_t* h_twin, int64_t n_tri, int64_t* h_off_out,
                                     int32_t* h_vtx_out, int64_t* id);
int64_t polylla_server_poll(polylla_server_t server, polylla_result* out, int64_t cap,
                            int64_t wait_us);
/*
 * polylla_server_cancel: a request still queued (not yet admitted) is removed and
 * completes at once with POLYLLA_ERR_CANCELLED (it is returned by the next poll);
 * its host buffers are no longer used when the call returns.  A request already
 * admitted, completed or unknown gives POLYLLA_ERR_STATE and runs to its end.
 */
polylla_status polylla_server_cancel(polylla_server_t server, int64_t id);
polylla_status polylla_server_info(polylla_server_t server, polylla_server_stats* out);
polylla_status polylla_server_destroy(polylla_server_t server);

/*
 * Failure injection for tests: the k-th device allocation the library makes from
 * now on (counting every buffer of a handle, a batch or a server slot) fails as if
 * the device were out of memory; k <= 0 turns it off.  Host-side only: the
 * failing call returns before reaching the device.  Each entry point must then
 * return POLYLLA_ERR_OOM (a served request: complete with it) and free what it
 * had allocated.
 */
void polylla_debug_fail_alloc(int64_t k);

/*
 * Test switch (Section 3.2.3's split, its rarer device paths): with enable != 0,
 * the reparation of this handle takes the paths normally kept for polygons with
 * a repeated vertex on every polygon -- one-tip pieces by chasing the successors
 * (counted in n_one_chase), several-tip pieces ordered by (origin, half-edge) with
 * half-edges found by turning (n_multi_turn), and each split's far node found
 * through turn(oj) -- so that tests can compare those paths with the oracle on any
 * mesh.  The polygons are the same either way.  While it is on, polylla_run
 * takes the multi-kernel path at every mesh size.  Errors:
 * POLYLLA_ERR_INVALID_ARG for a null handle.
 */
polylla_status polylla_debug_rare_paths(polylla_mesh_t mesh, int enable);

/*
 * Test switch (Section 3.2.3's order of splits, in the one-block path of
 * polylla_run): with enable != 0, every polygon with tips is split piece by piece
 * as the rule states it -- the first piece with a tip at its smallest tip, the
 * piece re-walked after each split -- instead of all its tips in increasing
 * order with the pieces ordered afterwards (the form the path takes when its
 * scratch holds the polygon's lists), so that tests can compare both forms with
 * the oracle.  The polygons are the same either way.  Errors:
 * POLYLLA_ERR_INVALID_ARG for a null handle.
 */
polylla_status polylla_debug_split_by_pieces(polylla_mesh_t mesh, int enable);

#ifdef __cplusplus
}
#endif
#endif /* POLYLLA_H */
