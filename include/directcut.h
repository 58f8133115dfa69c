/*
 * directcut.h -- C ABI of libdirectcut.so, a GB300 (sm_103a) implementation of
 * the parallel direct cut of Crabill, Witherden & Jameson (arXiv 1711.07663).
 *
 * The operation (Sec. 4.2 "Parallel Direct Cut Algorithm" of the paper): every
 * element of a curved order-p hexahedral background grid computes its minimum
 * distance to a closed cut surface of order-q quadrilateral faces and is
 * classified as HOLE (inside the surface), FIELD (outside) or FRINGE (the
 * paper's "intersecting" status: distance <= tol).  Element faces and cut faces
 * are linearised into triangles (2 per sub-quad of the (p+1)^2 / (q+1)^2 node
 * grids, Fig. "quadsplit"), the element-surface distance is the minimum
 * triangle-triangle distance (Sec. 4.2, Alg. cp1/cp2 with tol = 1e-7), and the
 * side comes from the dot product of the minimal vector with the outward face
 * normal (Sec. 4.1/4.2), averaged over the faces that share the closest point.
 *
 * Also here: what follows the cut (the union of several cuts, the
 * artificial-boundary faces, the unblank step of a moving grid), the paper's
 * own truncating variant of the exact test (DC_HEURISTIC), a launch-shape
 * autotuner, and the donor search for receptor points (dc_pc_*).
 *
 * Conventions
 *   element nodes  float64 [n_elem][(p+1)^3][3]; node (i,j,k) at
 *                  i + (p+1)*(j + (p+1)*k), i along xi fastest (the tensor
 *                  product Lagrange nodes of Eq. (reftophys)).
 *   face nodes     float64 [n_faces][(q+1)^2][3]; node (i,j) at i + (q+1)*j.
 *                  dx/dxi x dx/deta must point OUT of the region to blank, and
 *                  the faces must form a closed, watertight surface (shared
 *                  nodes bit-identical).
 *   pose           12 float64, row-major [R | t]: x' = R x + t applied to every
 *                  face node before the cut (rigid motion of the body, Sec. 4.3).
 *   flags          int8 per element: DC_HOLE 0, DC_FIELD 1, DC_FRINGE -1.
 *   dist           float64 per element: +d (FIELD), -d (HOLE), d (FRINGE) for
 *                  elements that reach the exact test; elements decided by the
 *                  Cartesian hole map (Sec. 4.2, "hole maps") get -HUGE_VAL
 *                  (hole) or +HUGE_VAL (field).
 *
 * Ownership: the caller owns every pointer it passes.  dc_create copies the
 * meshes to the device.  dc_cut reads the request's inputs before it returns.
 * dc_submit uploads host face nodes to the device (and copies the pose)
 * before it returns, so the caller may overwrite them at once; device face
 * nodes are read by the cut on the GPU and must stay unchanged until dc_poll
 * reports completion.  Output buffers must stay valid until dc_cut returns, or
 * until dc_poll reports completion of a submitted ticket.
 *
 * Errors: no exception crosses this ABI.  Every call returns a dc_status; the
 * text of the calling thread's last error is available from dc_last_error().
 *
 * Threads: calls on one context are serialised by the context; several
 * contexts may be used from several threads.
 */
#ifndef DIRECTCUT_H
#define DIRECTCUT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dc_ctx dc_ctx;
typedef int32_t dc_status;

enum {
    DC_OK = 0,
    DC_PENDING = 1,      /* dc_poll: not finished yet */
    DC_EINVAL = -1,      /* invalid argument (orders, counts, NaN nodes, pointers) */
    DC_ENOMEM = -2,      /* device or host allocation failed */
    DC_ECUDA = -3,       /* a CUDA runtime call failed */
    DC_EBUSY = -4,       /* no serving slot / memory budget free: retry later */
    DC_ETIMEDOUT = -5,   /* dc_poll: timeout elapsed, or a device wait ran out */
    DC_ENOTFOUND = -6,   /* unknown mesh index or ticket */
    DC_ECANCELED = -7,   /* the context was destroyed with the ticket in flight */
    DC_EINTERNAL = -8    /* a device-side capacity was exceeded (message says which) */
};

enum { DC_HOLE = 0, DC_FIELD = 1, DC_FRINGE = -1 };

/* Precision of the bulk triangle-triangle tests (Sec. 4.2 remarks that the
 * prepass may use single precision).  DC_FP32_RECHECK evaluates all candidate
 * pairs in FP32 with certified error bounds and re-solves, in FP64, only the
 * pairs whose FP32 lower bound lies within the bound of the best distance;
 * DC_FP64 evaluates every pair in FP64.  Both give the same flags.
 *
 * DC_HEURISTIC is the paper's own truncating variant instead of the exact
 * test (Sec. 4.2, Alg. cp0-cp2): per candidate, the 16 faces with the smallest
 * OBB-box key, the 4 with the smallest corner-triangle distance, and the
 * element triangles of the three faces at the nearest corner.  Its flags can
 * differ from the exact ones (a fringe element whose nearest faces fall
 * outside the 16 or 4 is reported hole or field); each of its decisions is
 * taken as in FP64.  dist_out holds its (upper-bound) distance. */
enum { DC_FP64 = 0, DC_FP32_RECHECK = 1, DC_HEURISTIC = 2 };

typedef struct {
    int32_t p;                /* element order, 1..4 */
    int64_t n_elem;           /* >= 1 */
    const double *nodes;      /* [n_elem][(p+1)^3][3] */
    int32_t nodes_on_device;  /* 0: host pointer, 1: device pointer (both copied) */
} dc_mesh_desc;

typedef struct {
    int32_t device;           /* CUDA device ordinal */
    int32_t precision;        /* DC_FP32_RECHECK (default), DC_FP64 or DC_HEURISTIC */
    size_t mem_budget_bytes;  /* device bytes the context may hold; 0 = no limit */
    double tol;               /* fringe tolerance, absolute mesh units; 0 -> 1e-7 (Alg. cp1) */
    int32_t holemap_cells;    /* hole-map cubes along the longest surface side, 8..80;
                                 0 -> automatic: about 1.8 cubes per mean element edge of
                                 the cut grid, 16..80 (the paper uses 60-80) */
    int32_t bin_cubes;        /* hole-map cubes per face bin along each axis, 1..16; 0 -> 4 */
    int32_t max_inflight;     /* serving slots for dc_submit, 1..64; 0 -> 4 */
    int32_t profile;          /* 1: time each phase with CUDA events (dc_get_stats) */
    int32_t reserve_faces;    /* dc_create sizes every slot's device arena and pinned
                                 staging (instance records, counters, host flags) for
                                 one request of this many
                                 order-2 faces on the largest mesh, from one device block
                                 and one pinned block, so such requests never allocate
                                 (larger ones, and the first dc_submit with host
                                 distances, grow the slot first); 0 -> 8192, -1 ->
                                 reserve nothing (grow on first use).  A reservation
                                 that would exceed mem_budget_bytes is skipped. */
} dc_config;

typedef struct {
    int32_t q;                /* face order, 1..4 */
    int64_t n_faces;          /* >= 1 */
    const double *face_nodes; /* [n_faces][(q+1)^2][3] */
    const double *pose;       /* host pointer to 12 doubles [R|t], or NULL (identity) */
    int8_t *flags_out;        /* [n_elem] */
    double *dist_out;         /* [n_elem] or NULL */
    int32_t on_device;        /* 1: face_nodes, flags_out, dist_out are device pointers */
    int32_t async;            /* dc_cut only, device pointers only: 1 = return after
                                 enqueueing on `stream`; results are valid once the
                                 stream reaches that point */
    void *stream;             /* cudaStream_t for dc_cut; NULL = the context's stream */
    float *fp32_dist_out;     /* optional [n_elem], DC_FP32_RECHECK with dist_out only, dc_cut /
                                 dc_cut_batch only: each exact-test element's distance as the
                                 FP32 bulk alone computed it (the smallest FP32 triangle-pair
                                 distance, signed as dist_out) before any FP64 re-solve, for
                                 reporting the FP32 error; NaN where the FP32 stage computed
                                 none (elements settled by their node labels, or redone in
                                 FP64), +-inf where the hole map decided.  Same memory kind
                                 as dist_out.  NULL: not written. */
} dc_request;

typedef struct {
    int64_t n_elem;           /* elements classified by the last dc_cut / dc_cut_batch */
    int64_t n_candidates;     /* elements the hole map could not decide (exact test) */
    int64_t n_fringe, n_hole, n_field;
    int64_t faces_visited;    /* element-face pairs whose triangles were tested */
    int64_t pairs_bulk;       /* triangle pairs evaluated in the bulk precision */
    int64_t pairs_recheck;    /* triangle pairs re-solved in FP64 */
    int64_t fallbacks;        /* elements redone in FP64 after a list overflow */
    int64_t holemap_rows_undecided; /* hole-map rows whose surface crossings could not be
                                       certified (their cubes are left "near") */
    float ms_surface;         /* profile=1 only: pose, face boxes, hole map, bins and the
                                 element classification (one fused kernel) */
    float ms_holemap;         /* 0: part of ms_surface (kept for the layout) */
    float ms_classify;        /* 0: part of ms_surface (kept for the layout) */
    float ms_exact;           /* exact element-face tests + sign (main pass) */
    float ms_redo;            /* FP64 pass over elements whose FP32 re-solve list overflowed
                                 (flags-only form: over its full-search list) */
    float ms_total;
    int64_t near_tasks;       /* flags-only requests: (element, face) pairs of boxes within
                                 tol listed for the flat exact test */
    int64_t n_full_search;    /* candidates decided by the full per-element search
                                 (distances requested, or no node labelled by the hole map) */
    int64_t near_pairs_full;  /* flags-only requests: listed triangle pairs that plane
                                 separation could not settle (full FP32 test) */
    int64_t heur_rescans;     /* DC_HEURISTIC: candidates whose FP32 key scan could not
                                 certify the 16 nearest faces (rescanned in FP64) */
    int64_t heur_resolves;    /* DC_HEURISTIC: faces whose pass-1 distance was re-solved
                                 in FP64 to order or zero it */
} dc_stats;

/* Fill *cfg with the defaults listed above. */
dc_status dc_config_default(dc_config *cfg);

/* Create a context on cfg->device holding n_meshes resident background grids
 * (copied; their element boxes are cached).  *out receives the context. */
dc_status dc_create(const dc_config *cfg, const dc_mesh_desc *meshes, int32_t n_meshes, dc_ctx **out);

/* Cut resident mesh `mesh` with one surface; synchronous unless req->async. */
dc_status dc_cut(dc_ctx *ctx, int32_t mesh, const dc_request *req);

/* Cut n (mesh, surface) instances in one batched launch sequence: every phase
 * runs once over all instances (persistent exact-test kernel over the union of
 * their candidates).  When every request leaves dist_out NULL the batch takes
 * the faster flags-only form of the exact stage; when any asks for distances
 * the whole batch takes the distance form (same flags either way).
 * Synchronous; requests must not set async. */
dc_status dc_cut_batch(dc_ctx *ctx, int32_t n, const int32_t *meshes, const dc_request *reqs);

/* Serving: admit a request into a free slot (DC_EBUSY when none is free or the
 * memory budget is exhausted), take its host inputs (host face nodes are
 * uploaded on the slot's stream and the call waits for that copy; the pose is
 * copied), enqueue the cut on the slot's stream and return a ticket.  Requests in different slots overlap on the GPU.  A request
 * within the slot's reservation (dc_config.reserve_faces) allocates nothing. */
dc_status dc_submit(dc_ctx *ctx, int32_t mesh, const dc_request *req, uint64_t *ticket);

/* Wait up to timeout_us (0 = just test, <0 = wait until done) for a ticket:
 * DC_OK when its outputs are written (the slot is released), DC_PENDING if
 * not done, or the error the cut ended with. */
dc_status dc_poll(dc_ctx *ctx, uint64_t ticket, int64_t timeout_us);

/* Counters and (profile=1) phase times of the last dc_cut / dc_cut_batch. */
dc_status dc_get_stats(dc_ctx *ctx, dc_stats *out);

/* Launch shapes of a context's cuts.  None of them changes a result: every
 * setting gives the same flags and distances, only the time differs.
 *   cubes_per_edge   hole-map cubes per mean element edge when holemap_cells is
 *                    0 (automatic), 0.5..4; 1.8 by default.  Finer maps leave
 *                    fewer candidate elements but cost more cubes per face.
 *   bin_cubes        hole-map cubes per face-bin side, 2..16 (at least
 *                    min(dc_config.bin_cubes, 2)); dc_config.bin_cubes by default.
 *   warps_per_cta    warps per block of the flags-only exact stage: 4, 8 or 16
 *                    (8 by default); lowered at launch to what the element and
 *                    face orders' shared memory allows.
 *   cands_per_warp   candidate elements a warp takes from the shared cursor at
 *                    once: 1, 2, 4 or 8 (1 by default).
 *   ms               dc_autotune: median time of the chosen setting; ignored
 *                    by dc_set_tuning. */
typedef struct {
    float cubes_per_edge;
    int32_t bin_cubes;
    int32_t warps_per_cta;
    int32_t cands_per_warp;
    float ms;
} dc_tuning;

/* The context's current launch shapes. */
dc_status dc_get_tuning(dc_ctx *ctx, dc_tuning *out);

/* Set the launch shapes of later cuts; DC_EINVAL (nothing changed) for a value
 * outside the ranges above. */
dc_status dc_set_tuning(dc_ctx *ctx, const dc_tuning *t);

/* Autotuner: run the batch (as dc_cut_batch) under every setting of the sweep
 *   cubes_per_edge {1.2, 1.8, 2.7} (only when holemap_cells is 0)
 *   x bin_cubes {2, 4, 8} x warps_per_cta {4, 8, 16} x cands_per_warp {1, 2, 4, 8},
 * one untimed run then `repeats` (1..50) runs timed by CUDA events on the
 * context's stream, keep the setting with the smallest median time, set it on
 * the context and run the batch once more with it, so the outputs hold its
 * result.  *best (may be NULL) receives the setting and its median time;
 * *n_trials (may be NULL) the number of settings timed.  Synchronous; the
 * requests must not set async.  On an error the previous setting stays. */
dc_status dc_autotune(dc_ctx *ctx, int32_t n, const int32_t *meshes, const dc_request *reqs, int32_t repeats,
                      dc_tuning *best, int32_t *n_trials);

/* Drain in-flight work, then free everything the context owns. */
void dc_destroy(dc_ctx *ctx);

/* Message of the calling thread's last failing call ("" if none).  Messages
 * are kept per thread, not per context: ctx may be NULL (as for the calls that
 * take no context), and a context used from several threads gives each thread
 * its own message. */
const char *dc_last_error(const dc_ctx *ctx);

/* Allocation-free cut, for callers that cannot allocate device memory at the
 * time they cut: real-time loops that forbid allocation after start-up
 * (cudaMalloc and cudaFree may block and synchronise the device, so their
 * latency has no bound) and hosts whose own allocator owns all device memory
 * (a caching pool that reserves the GPU's memory up front, where a second
 * allocator would fail or fragment it).  The paper has no counterpart; it is
 * the cut of dc_cut for one background grid, without a context.
 *
 *   nodes       device pointer, [n_elem][(p+1)^3][3] float64 (not copied)
 *   face_nodes  device pointer, [n_faces][(q+1)^2][3] float64
 *   pose        host pointer to 12 doubles [R|t], or NULL
 *   tol         fringe tolerance; 0 -> 1e-7
 *   flags_out   device pointer, [n_elem] int8 (required)
 *   dist_out    device pointer, [n_elem] float64, or NULL (flags only)
 *   stream      cudaStream_t to run on (NULL: the legacy default stream);
 *               the call returns after that stream has finished the cut.
 *
 * Every scratch buffer comes from one fixed 8 MiB array in the library's
 * device memory, which each GPU that loads the library holds until the
 * process exits; the call makes no cudaMalloc/cudaFree (nor any other
 * allocating call).  Sizes whose scratch does not fit are rejected with
 * DC_EINVAL and a message giving the bytes needed (40 bytes per element, about
 * 270 bytes per Q2 face or 660 per Q4 face, plus 2.6 MiB: 65,536 elements with
 * 8,192 Q2 faces fit).  The hole map uses 64 cubes on the longest side and 4-cube
 * face bins, the bulk tests FP32 with FP64 re-solve (flags identical to
 * dc_cut).
 *
 * All calls in a process share the array, which keeps the last call's
 * contents; each call resets what must start at zero.  Calls are serialised
 * by a lock in the library, and each returns only after its stream has
 * finished (on an error too, once work was queued), so two calls never use the
 * array at once; work on the array that overlapped on the GPU would race.
 *
 * The first call on a device sets up (looks up the array's device address,
 * uploads the triangle tables, sets kernel attributes) with that device
 * current. */
dc_status dc_cut_noalloc(int32_t p, int64_t n_elem, const double *nodes, int32_t q, int64_t n_faces,
                         const double *face_nodes, const double *pose, double tol, int8_t *flags_out,
                         double *dist_out, void *stream);

/* ---------------------------------------------------------------------------
 * After the cut: several cutting surfaces, artificial-boundary faces, and the
 * unblank step of a moving grid (Sec. 4.2, final paragraphs; Algorithm
 * "Artificial Boundary unblank procedure", Sec. 3).  One cut removes its
 * DC_HOLE elements, and for a solid wall (DC_WALL) also its DC_FRINGE
 * elements; an overset boundary (DC_OVERSET) keeps the elements it passes
 * through.  iblank arrays are int8: 1 kept, 0 removed.  All arrays are device
 * pointers; the calls allocate nothing, run on `stream` (NULL: the legacy
 * default stream) and return after it has finished; counts are returned
 * through host pointers.  Calls are serialised by a lock in the library.
 * Errors: DC_EINVAL for NULL pointers, n_elem < 1 or an unknown kind,
 * DC_ECUDA if a CUDA call fails.
 * ------------------------------------------------------------------------- */
enum { DC_WALL = 0, DC_OVERSET = 1 };

/* iblank_out[e] = 0 if any of the n_cuts (1..8) cuts removes element e, else 1.
 * flags: host array of n_cuts device pointers to int8 flag arrays [n_elem]
 * (the output of dc_cut); kinds: host array of n_cuts DC_WALL / DC_OVERSET. */
dc_status dc_blank_union(int32_t n_cuts, const int8_t* const *flags, const int32_t *kinds, int64_t n_elem,
                         int8_t *iblank_out, void *stream);

/* Artificial-boundary faces: ab_mask[e] has bit j (faces 0..5: xi = -1, +1,
 * eta = -1, +1, zeta = -1, +1) set when element e is kept and its neighbour
 * across face j is removed.  neighbours: [n_elem][6] int64 element indices,
 * -1 where a face has no neighbour.  *n_ab receives the number of such faces. */
dc_status dc_ab_faces(int64_t n_elem, const int8_t *iblank, const int64_t *neighbours, uint8_t *ab_mask,
                      int64_t *n_ab, void *stream);

/* The unblank step for one cut kind: flags_t and flags_tp are the cuts at the
 * current time and at t + dt; iblank_prev the blanking of the previous step.
 * Wall: removed now if removed by either cut; overset: if removed by both.
 * iblank_out receives the new blanking, unblank_out[e] = 1 for the elements
 * removed before and kept now (to be filled by interpolation), *n_unblank
 * their number. */
dc_status dc_unblank(int32_t kind, int64_t n_elem, const int8_t *iblank_prev, const int8_t *flags_t,
                     const int8_t *flags_tp, int8_t *iblank_out, uint8_t *unblank_out, int64_t *n_unblank,
                     void *stream);

/* Library version string. */
const char *dc_version(void);

/* Allocation accounting and failure injection, for testing the handling of
 * DC_ENOMEM without exhausting memory.  Every device allocation (cudaMalloc)
 * and pinned host allocation (cudaMallocHost) the library makes, in any
 * context or thread, is counted.  after >= 0 arms a one-shot failure: the
 * allocation `after` allocations from now (0: the next one) reports failure
 * as if memory were exhausted, and the call that made it returns DC_ENOMEM
 * after releasing what it holds; the context stays usable.  after < 0
 * disarms.  Returns the number of allocations made since the library was
 * loaded (before this call).  Host-side only: no GPU memory is touched and
 * no device is needed. */
int64_t dc_fail_alloc(int64_t after);

/* ------------------------------------------------------------------------
 * Point connectivity: donors for receptor points (after the cut)
 * ------------------------------------------------------------------------
 * Sec. "Donor/Receptor Point Connectivity on GPUs": the flux points of the
 * artificial-boundary faces of one grid need a donor element of another grid
 * and their reference coordinates in it.  dc_pc_create builds, once, a
 * balanced search tree over the donor grid's element boxes on the host (one
 * element per node, median splits over the six box coordinates in turn, as
 * an alternating digital tree) and copies it with the grid to the device.
 * The grid may then move rigidly: dc_pc_locate takes each point into the
 * grid's initial frame with the inverse of `pose` instead of rebuilding the
 * tree, finds the elements whose node box holds it by a depth-first traversal
 * with a fixed stack (32 entries), and checks them in index order with the
 * clamped Newton inversion of the isoparametric map (Eq. ref-update: from
 * xi = 0, xi clamped to [-1 - 1e-4, 1 + 1e-4], at most 10 FP32 steps in the
 * element frame, then FP64 steps on the original nodes).  A point's donor is
 * the first (lowest-index) element where the residual falls to 1e-10 h (h:
 * the element box's largest side) with max |xi_a| <= 1 + 1e-8; otherwise -1.
 * Lagrange nodes are equispaced on [-1, 1] (tensor order, xi fastest). */
typedef struct dc_pc dc_pc;

typedef struct {
    int64_t n_points;         /* points of the last dc_pc_locate */
    int64_t n_found;          /* ... with a donor */
    int64_t candidates;       /* element boxes that held a point (Newton solves tried) */
    int64_t fp64_steps;       /* FP64 Newton steps after the FP32 stage */
    int64_t tree_depth;       /* levels of the search tree */
} dc_pc_stats;

/* Copy a donor grid of n_elem order-p hexes (p 1..4; nodes [n_elem][(p+1)^3][3],
 * host or device pointer) to `device` and build its search tree.  DC_EINVAL
 * for bad sizes or a non-finite node. */
dc_status dc_pc_create(int32_t device, int32_t p, int64_t n_elem, const double *nodes, int32_t nodes_on_device,
                       dc_pc **out);

/* Donors of n_pts points pts [n_pts][3] (world frame).  pose: 12 doubles
 * [R|t], the grid's rigid motion from its initial frame (NULL: none).
 * donor_out [n_pts] (-1: no donor), ref_out [n_pts][3] reference coordinates
 * (0 when none).  on_device: all three arrays are device pointers (else host).
 * Synchronous on `stream` (NULL: the context's own).  DC_EINTERNAL when a
 * point lies in more than 16 element boxes (its answer is then incomplete). */
dc_status dc_pc_locate(dc_pc *pc, int64_t n_pts, const double *pts, const double *pose, int64_t *donor_out,
                       double *ref_out, int32_t on_device, void *stream);

/* Counters of the last dc_pc_locate. */
dc_status dc_pc_get_stats(dc_pc *pc, dc_pc_stats *out);

/* Free the donor grid and its tree. */
void dc_pc_destroy(dc_pc *pc);

#ifdef __cplusplus
}
#endif

#endif /* DIRECTCUT_H */
