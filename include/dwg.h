/*
 * dwg.h -- C ABI of the Diffusing Winding Gradients engine (libdwg.so).
 *
 * The engine orients an unoriented point cloud by the iteration of the
 * paper's Algorithm 1 (Diffusing Winding Gradients, arXiv 2405.13839,
 * Sec. 4.3):
 *   1. evaluate the generalized winding number w and its gradient at every
 *      input point, and w at the corners of the leaves of an octree of depth
 *      d around the cloud (Sec. 3 Eq. 2/3; screened variant Sec. 4.2 Eq. 5);
 *   2. take the iso-value w_bar as the mean of w over the input points
 *      (Eq. 6, averaged over the inputs as in the abstract and Sec. 4.1);
 *   3. extract the w_bar level set in every leaf, give each face the
 *      gradient from its cross product, add it to the face's k nearest input
 *      points and normalise (Eq. 7);
 *   4. stop when the mean of the largest 1% of the per-point normal changes
 *      is at most tol degrees (Sec. 5.1, "Model-independent Parameters").
 * Around it, the options of Sec. 5.1-5.2: local-Voronoi area weights
 * (dwg_voronoi_weights), random, PCA, Gauss-map, given or learned initial
 * normals (dwg_set_init), the modified Poisson kernel with per-point clamp
 * radii (dwg_set_regularization), exact or Barnes-Hut evaluation
 * (dwg_set_tree); and the outputs: the normals (dwg_orient) and the w_bar
 * level set as triangles (dwg_extract_level_set).
 * Every step runs in this library's CUDA kernels on one GPU; there is no CPU
 * fallback.  A call that needs the GPU and finds none returns DWG_ERR_CUDA.
 *
 * Conventions for every function below:
 *   - Return value: DWG_OK (0), DWG_NOT_CONVERGED (1, informational), or a
 *     negative DWG_ERR_* code; dwg_last_error() then describes the failure.
 *   - Pointer arguments may be host memory (pageable or pinned) or device
 *     memory of the handle's device; the library tells them apart with
 *     cudaPointerGetAttributes.  The caller keeps ownership of every buffer
 *     it passes; the library copies what it needs and never frees it.
 *   - Point arrays are float32, n x 3, row-major (x, y, z per point), in the
 *     caller's units: no implicit normalisation, so rotations and
 *     translations of the input rotate and translate every result.
 *   - All GPU work is issued on the handle's stream (dwg_set_stream), and
 *     every function returns only after its results are in the caller's
 *     buffers.
 *   - A handle is not thread-safe; distinct handles are independent.
 */
#ifndef DWG_H
#define DWG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DWG_OK 0
#define DWG_NOT_CONVERGED 1
#define DWG_ERR_INVALID (-1)   /* bad argument or size */
#define DWG_ERR_CUDA (-2)      /* CUDA error or no usable GPU */
#define DWG_ERR_OOM (-3)       /* device allocation failed */
#define DWG_ERR_NONFINITE (-4) /* NaN or Inf in an input */
#define DWG_ERR_TIMEOUT (-5)   /* a bounded device-side wait gave up */
#define DWG_ERR_STATE (-6)     /* call not valid in the handle's state */

/* GWN kernels: plain Poisson kernel (Eq. 3) or screened (Eq. 5). */
#define DWG_KERNEL_PLAIN 0
#define DWG_KERNEL_SCREENED 1

/* Normal update: the level-set rule of Eq. 7 (default), or the point form
 * n_i <- -grad w(p_i) / |grad w(p_i)| (a reading of Eq. 4 kept for study). */
#define DWG_UPDATE_LEVELSET 0
#define DWG_UPDATE_DIRECT 1

/* Initial normals (Sec. 5.1): uniform random directions drawn on the
 * device from a seed, or caller-given normals. */
#define DWG_INIT_RANDOM 0
#define DWG_INIT_GIVEN 1
#define DWG_INIT_LEARNED 2
#define DWG_INIT_PCA 3
#define DWG_INIT_GAUSS 4

/* Evaluation path: exact all-pairs sums, or the Barnes-Hut far field of
 * Sec. 5.2; AUTO takes all-pairs up to 65,536 points and the tree above
 * (dwg_autotune can choose by measurement instead). */
#define DWG_PATH_AUTO 0
#define DWG_PATH_ALLPAIRS 1
#define DWG_PATH_TREE 2

typedef struct dwg_ctx *dwg_handle;

/*
 * Create a handle for a cloud of n >= 1 points (float32 n x 3, host or
 * device).  Copies the points to the current CUDA device, checks them for
 * NaN/Inf (DWG_ERR_NONFINITE), sorts them along a Morton curve and builds
 * the spatial structures that depend on positions only.  Area weights
 * default to a_i = 1 (Sec. 5.1, "Computing Area Weights").  Default
 * parameters: plain kernel, eps = 0.5 * L / sqrt(n) with L the largest
 * bounding-box extent, no screening, 30 iterations, tol 0.1 degrees
 * (Sec. 5.1), octree depth 8, k = 10 (Sec. 5.1), level-set update, random
 * initialisation with seed 1.  On failure *out is NULL.
 */
int dwg_create(const float *points, int64_t n, dwg_handle *out);

/* Release every device resource of the handle.  NULL is ignored. */
void dwg_destroy(dwg_handle h);

/* Text of the last failure on this handle, or, when h is NULL, of the last
 * failed call that takes no handle (dwg_create, dwg_eval_w_noalloc).  Valid
 * until the next call on the handle. */
const char *dwg_last_error(dwg_handle h);

/* Issue all further work of the handle on this cudaStream_t (NULL: the
 * library's own stream).  The stream must belong to the handle's device. */
int dwg_set_stream(dwg_handle h, void *stream);

/*
 * Method parameters.
 *   kernel:    DWG_KERNEL_PLAIN or DWG_KERNEL_SCREENED.
 *   eps:       softening length > 0, in the caller's length unit: every
 *              kernel term uses rho^2 = |p - q|^2 + eps^2, the paper's
 *              "small constant added to the denominator" (Sec. 3).
 *   screening: lambda >= 0 of Eq. 5, in 1 / length^2; ignored for PLAIN.
 *   max_iters: >= 1, iteration cap of dwg_orient.
 *   tol:       > 0, convergence threshold in degrees (Sec. 5.1 uses 0.1).
 */
int dwg_set_params(dwg_handle h, int kernel, float eps, float screening, int max_iters,
                   float tol);

/*
 * Convergence rule of dwg_orient (tol from dwg_set_params, in degrees).
 *   DWG_CONV_TOP1 (default): the mean of the ceil(n / 100) largest per-point
 *     changes of the normal (angles) is at most tol (Sec. 5.1,
 *     "Model-independent Parameters").
 *   DWG_CONV_MEAN: the mean over all points of |n_new - n_old| is at most
 *     2 sin(tol / 2), the chord of an angle of tol (the measure the paper
 *     plots in Fig. 6).  Noise and outliers keep a few points moving by
 *     degrees long after the rest has settled, so the top-1 % rule may not
 *     be met within max_iters on such clouds.
 */
#define DWG_CONV_TOP1 0
#define DWG_CONV_MEAN 1
int dwg_set_convergence(dwg_handle h, int rule);

/*
 * The kNN scatter of Eq. 7 (not a parameter of the paper; results do not
 * depend on it).  A face whose cell has no candidate list searches the
 * points' bucket tree in its own thread; a face that is about as far from
 * many points as from its nearest (a level set far from the cloud, as near
 * the centre of a sphere) can make that search nearly exhaustive and hold
 * the whole launch.  A search that takes more than `budget` node visits and
 * point distances stops and hands the face to a second launch in which a
 * block of threads finishes it; the k points found, and so the sums, are the
 * same bits either way.  budget >= 0 (default 16384), or -1: every face
 * searches alone.  Batch handles apply it to every cloud.
 */
int dwg_set_knn_budget(dwg_handle h, int budget);

/*
 * Compensation of the exact all-pairs evaluator's sums of the Eq. 2/3 and
 * Eq. 5 terms, which are computed in FP32 here (the paper states no
 * precision and has no counterpart to this switch).  on = 1 (the
 * default): each thread sums 128 sources in plain FP32 and folds that tile
 * sum into a two-sum (hi, lo) pair; on = 0: the tile sums are added in plain
 * FP32 instead.  The switch exists to measure what the compensation buys
 * against the FP64 oracle; it applies to the all-pairs evaluator's default
 * shapes, softened kernel (the modified kernel and the Barnes-Hut path keep
 * their compensated sums).  Batch handles: DWG_ERR_STATE.
 */
int dwg_set_compensation(dwg_handle h, int on);

/*
 * How a batch handle (dwg_create_batch) runs an iteration of all its clouds
 * (the paper orients one cloud; batching is this library's).
 *   lanes in [1, DWG_MAX_BATCH_LANES] (default 1): batched phases.  The
 *     clouds are split into min(lanes, clouds) groups of about equal work;
 *     within a group every phase of the iteration -- Barnes-Hut moments per
 *     tree level, list evaluations, reduce, iso-value, level set, kNN
 *     scatter, update, the convergence select -- is one launch over all the
 *     group's clouds, and the groups run concurrently as branches of the
 *     iteration graph.  The launches per iteration grow with the lanes and
 *     the deepest tree, not with the number of clouds.
 *   lanes = 0: each cloud's chain of launches is a branch of the iteration
 *     graph on its own stream.
 * Every mode gives every cloud the same bits as orienting it alone.  The
 * batched phases need k = 10 and the softened kernel in every cloud;
 * otherwise the per-cloud branches run.  Not a batch handle: DWG_ERR_STATE;
 * lanes out of range: DWG_ERR_INVALID.
 */
#define DWG_MAX_BATCH_LANES 16
int dwg_set_batch_mode(dwg_handle h, int lanes);

/*
 * Discretisation and update rule.
 *   depth: octree depth d in [1, 14] (Sec. 5.1 recommends 8-10 up to 1M
 *          points, 11-13 beyond).
 *   knn:   k of Eq. 7's face-to-point assignment, in [1, 32] (paper: 10).
 *   mode:  DWG_UPDATE_LEVELSET or DWG_UPDATE_DIRECT.
 */
int dwg_set_update(dwg_handle h, int depth, int knn, int mode);

/*
 * Evaluation path and opening angle (Sec. 5.2 "Octree Traversal").
 *   path:  DWG_PATH_AUTO, DWG_PATH_ALLPAIRS or DWG_PATH_TREE.
 *   theta: opening angle in (0, 1]: a node of area-weighted centre c and
 *          radius r stands for its points as one dipole (its area-weighted
 *          normal sum at c) for a query q with |q - c| > r / theta, else it
 *          opens; leaves (16 Morton-consecutive points by default, see
 *          dwg_set_tuning) are summed exactly.
 *          The paper opens when |q - c| <= 2.3 r, i.e. theta = 1 / 2.3.
 * Default: AUTO, theta = 0.5.
 */
int dwg_set_tree(dwg_handle h, int path, float theta);

/*
 * Near-field regularisation of the kernel.
 *   DWG_REG_SOFTEN (default): rho^2 = |p_j - q|^2 + eps^2 with the eps of
 *     dwg_set_params (the paper's "small constant added to the denominator",
 *     Sec. 3, read as Plummer softening).
 *   DWG_REG_CLAMP: the modified Poisson kernel of Sec. 5.2 ("Poisson
 *     Kernels"): rho = max(|p_j - q|, delta_j) with a radius per source and no
 *     softening; inside the radius the term is <m_j, p_j - q> / delta_j^3
 *     (times F(delta_j) when screened) and its gradient -m_j F / delta_j^3.
 *     delta_j = the mean distance from p_j to those of its k nearest other
 *     points (ties by smaller input index) whose distance lies in
 *     [vmin, vmax]; if none does, the mean of all k distances clamped to
 *     [vmin, vmax].  The paper uses k = 10, vmin = 0.0015, vmax = 0.015 in
 *     its unit-box coordinates; vmin = vmax = 0 selects those values times
 *     the largest extent of the points' bounding box.
 *     Whether a pair lies inside is decided in float32 (|p_j - q|^2 from
 *     float offsets against delta_j^2 rounded to float).
 *     On the Barnes-Hut path a node opens unless the query is farther than
 *     both r / theta and r + (the largest radius of its points) from its
 *     centre, so far nodes never hold a point whose radius reaches the query
 *     and keep the unclamped dipole; leaf points take the clamp.  The group
 *     lists and the per-query walk implement it (without group lists, i.e.
 *     when they do not fit in memory, the per-query walk serves).
 *     dwg_autotune returns DWG_ERR_STATE while it is set (one evaluator
 *     shape; set the tree's settings by hand).  Batch handles refuse it
 *     (DWG_ERR_STATE).
 *   k: [1, 31] (CLAMP only).  delta_out: float32 n, input order, host or
 *   device, receives delta_j; may be NULL.
 */
#define DWG_REG_SOFTEN 0
#define DWG_REG_CLAMP 1
int dwg_set_regularization(dwg_handle h, int mode, int k, float vmin, float vmax,
                           float *delta_out);

/*
 * The w_bar level set of the handle's current normals as a triangle mesh
 * (Alg. 1's Marching Cubes step; the level set the method outputs beside the
 * normals).  With the handle's path and settings: w at the input points and
 * w_bar = their mean (FP64), w at the corners of the octree leaves of the
 * dwg_set_update depth (built if needed, in either update mode), then per
 * leaf the six-tetrahedron marching tetrahedra of the iteration: a cut
 * tetrahedron gives one triangle (one or three corners above w_bar) or two
 * (two above), with vertices at the linear-interpolation points of its cut
 * edges, wound so that (v1 - v0) x (v2 - v0) points toward decreasing w
 * (outward for outward normals).  Leaves of different sizes are not
 * stitched (no crack fixing).
 *   tri_out: float32 cap x 9 (x0 y0 z0 x1 y1 z1 x2 y2 z2), host or device, or
 *            NULL to count only; order unspecified.
 *   *count:  the number of triangles, written in every case; when it exceeds
 *            cap nothing else is written.
 *   iso_out: (host, may be NULL) w_bar.
 * The iteration state is reset (as by the next dwg_orient).  Batch handles:
 * DWG_ERR_STATE.
 */
int dwg_extract_level_set(dwg_handle h, float *tri_out, int64_t cap, int64_t *count,
                          double *iso_out);

/*
 * FP32 issue microbenchmarks of a device (not in the paper): the measured
 * denominators of the evaluators' roofline.  ffma_lane_ops_per_s: FP32 lane
 * operations per second of packed fused multiply-adds (fma.rn.f32x2; one
 * packed instruction = 2 lane operations), 8 independent chains per thread,
 * 8 CTAs of 256 threads per SM; rsqrt_per_s and ex2_per_s: MUFU reciprocal
 * square roots and base-2 exponentials (the screened kernel's factor) per
 * second, the same way.  Each is the faster of two timed launches of a few
 * milliseconds after a warm-up.  Returns DWG_ERR_INVALID for a bad device or
 * NULL outputs, DWG_ERR_CUDA on a CUDA error.
 */
int dwg_measure_fp32_peaks(int device, double *ffma_lane_ops_per_s, double *rsqrt_per_s,
                           double *ex2_per_s);

/*
 * Failure-detection self-check (not in the paper).  Every device-side wait of
 * the library (bulk-copy mbarriers, tensor-core commits) gives up after a
 * bounded number of polls, records the timeout in the handle's error flag
 * and lets the kernel return, so a stalled copy surfaces as DWG_ERR_TIMEOUT
 * on the host with the context intact.  This call exercises that path: one
 * CTA waits, through the evaluators' bounded wait, on an mbarrier that
 * expects an arrival nothing sends, for `polls` polls (in [1, 2^20]); it
 * returns DWG_ERR_TIMEOUT, clears the flag, and the handle stays usable.
 */
int dwg_selfcheck_wait(dwg_handle h, int polls);

/* Area weights a_i > 0 (float32, n, input order, host or device). */
int dwg_set_weights(dwg_handle h, const float *a);

/*
 * Local-Voronoi area weights (Sec. 5.1, "Computing Area Weights"; the paper
 * uses m = 15), computed on the device and installed as the handle's a_i.
 * For each point p_i: its m nearest other points (ties by smaller input
 * index; coincident copies count); the tangent plane through p_i whose
 * normal is the smallest-eigenvalue eigenvector of the covariance of p_i and
 * those neighbours (FP64); the neighbours projected onto it as the seeds of a
 * 2D Voronoi diagram (a seed projecting onto p_i imposes nothing); a_i = the
 * area of p_i's cell cut to the disk of radius half the largest projected
 * neighbour distance (the cut bounds the cells of points on the hull of
 * their neighbourhood and leaves interior cells of even samplings whole).
 * A neighbourhood with no extent takes the mean of the other areas (1, the
 * paper's default weight, when no area is positive).
 *   m:     in [3, 31].
 *   a_out: float32 n (input order, host or device) receives the weights; may
 *          be NULL.
 * On a batch handle every cloud gets its own weights (a_out in the input
 * layout).  Errors: DWG_ERR_INVALID (m), DWG_ERR_CUDA.
 */
int dwg_voronoi_weights(dwg_handle h, int m, float *a_out);

/*
 * Initial normals for the next dwg_orient.  DWG_INIT_RANDOM draws uniform
 * unit vectors from the splitmix64 stream (seed, 7): with u0, u1 the
 * uniforms 2i and 2i+1 (top 53 bits * 2^-53), z = 1 - 2 u0,
 * phi = 2 pi u1, n = (sqrt(1 - z^2) cos phi, sqrt(1 - z^2) sin phi, z);
 * normals is ignored.  DWG_INIT_GIVEN copies normals (float32 n x 3, input
 * order, host or device; each is normalised -- a vector of unit length to
 * within 4e-7 is taken as is, so normals from dwg_get_normals or dwg_orient
 * resume an orientation exactly (checkpoint / resume) -- zero vectors
 * rejected).
 * DWG_INIT_LEARNED (a project extension, not in the paper): `normals` points
 * to the 12,675 float32 parameters of the kNN-patch network (layout in
 * dwg_mlp_forward); the initial normal of each point is the normalised
 * network output for its patch features (dwg_mlp_features); where the output
 * is zero or not finite the random normal from `seed` is kept.
 * DWG_INIT_PCA (Sec. 5.1, "Normal Initialization"): the eigenvector of the
 * smallest eigenvalue of the covariance of the 10 nearest input points (the
 * point itself included; ties by smaller input index), computed in FP64 on
 * the offsets from the point; PCA gives the line, and the direction is the
 * one pointing away from the centre c of the bounding box (n . (p - c) > 0,
 * the Gauss map's side; where that is 0: n_z > 0, then n_y > 0, then
 * n_x > 0).  Where the covariance is zero (coincident points) the random
 * normal from `seed` is kept.  normals is ignored.
 * DWG_INIT_GAUSS (Sec. 5.1): n_i = (p_i - c) / |p_i - c| in FP64, c the centre
 * of the points' bounding box (the paper's models sit in a box centred at the
 * origin); a point at c keeps the random normal from `seed`.  normals is
 * ignored.
 */
int dwg_set_init(dwg_handle h, int mode, uint64_t seed, const float *normals);

/*
 * Run Algorithm 1 from the initial normals until convergence or max_iters.
 * normals_out (float32 n x 3, input order, host or device, may be NULL)
 * receives the final normals; *iters_out (may be NULL) the number of
 * iterations performed.  Returns DWG_NOT_CONVERGED if the cap was reached
 * (the normals are still written).  The whole loop runs on the device: one
 * CUDA graph launch whose conditional node repeats the iteration body.
 */
int dwg_orient(dwg_handle h, float *normals_out, int *iters_out);

/*
 * One iteration from the handle's current normals (the initial normals
 * before the first orient or step, else the latest ones), updating them.
 * Optional outputs in input order (each may be NULL, host or device):
 * w_out (n) and grad_out (n x 3) at the input points for the normals the
 * step started from; dtheta_out (n) the per-point change in degrees;
 * iso_out the iso-value w_bar; stat_out the convergence statistic.
 */
int dwg_step(dwg_handle h, float *w_out, float *grad_out, float *dtheta_out, double *iso_out,
             double *stat_out);

/* Current normals (float32 n x 3, input order). */
int dwg_get_normals(dwg_handle h, float *normals_out);

/* Replace the current normals (same layout); they become the initial
 * normals of the next dwg_step.  Zero vectors are rejected. */
int dwg_set_normals(dwg_handle h, const float *normals);

/*
 * w (and, if grad_out is not NULL, grad w) of the current oriented cloud at
 * m >= 1 arbitrary query points (float32 m x 3).  A query that coincides
 * exactly with input points skips those terms, as at the inputs.
 */
int dwg_eval_gwn(dwg_handle h, const float *queries, int64_t m, float *w_out,
                 float *grad_out);

typedef struct {
    int64_t n_points;
    int64_t n_leaves;        /* octree leaves at the current depth */
    int64_t n_corners;       /* distinct leaf corners (w query points) */
    int iters;               /* iterations of the last dwg_orient */
    int converged;
    int64_t faces_last;      /* level-set faces of the last iteration */
    double iso_last;         /* w_bar of the last iteration */
    double stat_last;        /* convergence statistic of the last iteration */
    double interactions;     /* kernel evaluations of the last dwg_orient */
    double ms_orient;        /* device time of the last dwg_orient */
    double interactions_eval; /* kernel evaluations of the last dwg_eval_gwn */
    double interactions_points_step;  /* dwg_profile_step: evaluations at the points */
    double interactions_corners_step; /* dwg_profile_step: evaluations at the corners */
    int kernels_per_iteration;        /* kernel launches in one iteration of the graph */
    int knn_deferred_last;   /* faces of the last iteration handed to a block (dwg_set_knn_budget);
                                beyond 65,536 the rest search alone */
} dwg_stats;

int dwg_get_stats(dwg_handle h, dwg_stats *out);

/* Per-iteration trace of the last dwg_orient: iso-value, convergence
 * statistic (degrees), mean |n_new - n_old|, face count.  Arrays of cap
 * entries (host memory, any may be NULL); *count receives the iterations. */
int dwg_get_trace(dwg_handle h, double *iso, double *stat, double *mean_dn, int64_t *faces,
                  int cap, int *count);

/*
 * Structures, for inspection and tests.
 * dwg_get_leaves: octree leaves at the current depth as int64 records
 *   (level, ix, iy, iz, nonempty), coordinates in units of the leaf's level,
 *   sorted by (level, ix, iy, iz); cap records at most (host or device).
 * dwg_get_corners: distinct leaf corners as sorted int64 keys
 *   X * (2^d + 1)^2 + Y * (2^d + 1) + Z in depth-d lattice units.
 * Both write *count (host) even when cap is too small (then nothing else).
 */
int dwg_get_leaves(dwg_handle h, int64_t *leaves_out, int64_t cap, int64_t *count);
int dwg_get_corners(dwg_handle h, int64_t *keys_out, int64_t cap, int64_t *count);

/*
 * Many clouds in one handle (the batched form of Alg. 1).
 * dwg_create_batch: points float32 (total x 3, host or device) with the
 *   clouds concatenated; offsets int64 (n_clouds + 1, host or device),
 *   offsets[0] = 0, offsets[n_clouds] = total, every cloud non-empty.  Each
 *   cloud gets its own root cube, octree, kNN tree, iso-value and
 *   convergence test; its default softening is its own (0.5 L / sqrt(n)) and
 *   its default octree depth is round(log2(n) / 2) clamped to [5, 10].
 *   dwg_set_params / dwg_set_update / dwg_set_tree / dwg_set_convergence on
 *   the batch handle apply to every cloud (dwg_set_params with eps = 0 keeps
 *   each cloud's own default softening); dwg_set_init takes every mode but
 *   DWG_INIT_GIVEN (cloud c uses seed + c).
 * dwg_orient_batch: runs every cloud until it converges (or max_iters); a
 *   converged cloud stops iterating while the others go on.  The whole loop
 *   is one CUDA graph launch; per iteration the all-pairs sums of every
 *   cloud on that path are one kernel launch.  normals_out (total x 3, host
 *   or device, may be NULL) in the input layout; iters_out (host, n_clouds,
 *   may be NULL).  Returns DWG_NOT_CONVERGED if any cloud reached the cap.
 * dwg_orient and dwg_step return DWG_ERR_STATE on a batch handle.
 */
int dwg_create_batch(const float *points, const int64_t *offsets, int n_clouds,
                     dwg_handle *out);
int dwg_orient_batch(dwg_handle h, float *normals_out, int *iters_out);

/*
 * Per-kernel device times of one iteration, for profiling.  Runs one
 * iteration exactly like dwg_step (same kernels, same launch shapes, on the
 * handle's stream) with a CUDA event pair around each launch, and writes the
 * elapsed milliseconds into ms_out (host, cap entries) in this fixed order:
 *   0 eval_points    w and grad w at the input points (all-pairs)
 *   1 reduce_points  combine the source-chunk partials, coincident terms
 *   2 iso            w_bar
 *   3 eval_corners   w at the octree leaf corners (all-pairs)
 *   4 reduce_corners combine the source-chunk partials
 *   5 mc_faces       level-set faces
 *   6 knn_scatter    face gradients to the k nearest points
 *   7 normal_update  new normals, per-point change
 *   8 select         convergence statistic
 * Entries 3-6 are 0 for DWG_UPDATE_DIRECT.  *count receives 9.
 */
int dwg_profile_step(dwg_handle h, float *ms_out, int cap, int *count);

/*
 * Learned warm start (a project extension; the paper initialises with
 * random, PCA or Gauss-map normals, Sec. 5.1).  The network maps a 64-value
 * patch feature row to 3 outputs: three hidden layers of 64 with ReLU,
 * bfloat16 weights and activations on the tensor cores, fp32 accumulation.
 * Parameters (float32, 12,675): W1[64][64] (out, in), b1[64], W2[64][64],
 * b2[64], W3[64][64], b3[64], W4[3][64], b4[3].
 *
 * dwg_mlp_features: feature rows of the handle's points (float32 n x 64,
 *   input order, host or device): offsets to the 16 nearest other points
 *   (exact, ascending, ties to the smaller index) divided by their RMS
 *   length, then (p - c) / R with c the centroid and R the RMS radius of
 *   the cloud, zero padding.
 * dwg_mlp_forward: Y (B x 3) = network(X) for B rows of X (B x 64).
 * dwg_mlp_grad: mean squared error (1/B) sum |network(X) - T|^2 of B rows
 *   against targets T (B x 3) into *loss (host) and its gradient with
 *   respect to every parameter into grad (12,675).
 * dwg_mlp_adam: one Adam step (beta1 0.9, beta2 0.999, eps 1e-8, step >= 1)
 *   of params with grad, moments m and v (12,675 each, updated in place).
 * The last three take DEVICE pointers only and run on `stream` (NULL: the
 * legacy default stream); they return after the results are written.
 */
int dwg_mlp_features(dwg_handle h, float *X_out);
int dwg_mlp_forward(const float *params, const float *X, int64_t B, float *Y, void *stream);
int dwg_mlp_grad(const float *params, const float *X, const float *T, int64_t B, float *grad,
                 double *loss, void *stream);
int dwg_mlp_adam(float *params, const float *grad, float *m, float *v, int step, float lr,
                 void *stream);

/*
 * Autotuner (a project extension; the paper sets its parameters by hand,
 * Sec. 5.1, and fixes the opening test at 2.3 r, Sec. 5.2).
 *
 * dwg_tuning: the performance settings of a handle.
 *   path:            DWG_PATH_ALLPAIRS or DWG_PATH_TREE (AUTO resolved);
 *   points_pairs, points_threads:   shape of the exact evaluator of w and
 *                    grad w at the points (query pairs per thread, CTA size);
 *   corners_pairs, corners_threads: shape of the exact evaluator of w at the
 *                    octree-leaf corners;
 *   tree_leaf:       points per Barnes-Hut leaf (16, 32, 64 or 128);
 *   theta:           opening angle of the Barnes-Hut path (as dwg_set_tree);
 *   tree_group:      0: the opening test per query (Sec. 5.2 as printed);
 *                    1 (default): per group of 64 consecutive queries,
 *                    against the group's bounding box -- conservative (far
 *                    for the box is far for each query), so every query's
 *                    error stays within its per-query bound; the groups'
 *                    interaction lists at the points and the leaf corners
 *                    are built once and evaluated every iteration;
 *   knn_lists:       1 (default): the faces' k-nearest-point searches (Eq. 7)
 *                    scan a candidate list per octree leaf cell, built once
 *                    per discretisation: the points within r_k(c) + 2 h of
 *                    the cell centre c (h the half-diagonal), which contain
 *                    the k nearest points of every position in the cell, so
 *                    the scan returns exactly the tree search's result; cells
 *                    with more than 256 candidates keep the tree search.
 *                    0: every face walks the bucket tree.  Not tuned
 *                    (dwg_autotune keeps the handle's value);
 *   w_err:           largest |w_tree - w_exact| the tuner saw on its sample
 *                    (0 for the exact path);
 *   ms_points, ms_corners: device time of one evaluation at the points and
 *                    at the corners with these settings (milliseconds);
 *   from_cache:      1 when dwg_autotune took the settings from its cache.
 *
 * dwg_autotune(h, what, w_budget, cache_path, out): measures on the handle's
 *   own cloud, current normals and stream.  what = DWG_TUNE_SHAPES (every
 *   compiled evaluator shape, timed with CUDA events, median of three) and/or
 *   DWG_TUNE_TREE (per leaf size and test form, the largest opening angle in
 *   {0.9, 0.8, ..., 0.2} whose w differs from the exact all-pairs w by at most
 *   w_budget (absolute) on a sample of up to 2,048 points and 2,048 corners
 *   (runs of 64 consecutive ones, spread evenly);
 *   then the fastest of those).  With path DWG_PATH_AUTO the faster path that meets
 *   the budget is chosen; with DWG_PATH_TREE and no angle meeting the budget
 *   the call fails with DWG_ERR_INVALID.  The chosen settings are applied to
 *   the handle and written to *out (may be NULL).  cache_path (may be NULL):
 *   a text file with one JSON object per line, keyed by the GPU's name and SM
 *   count and the problem (sizes, kernel, screening, update rule, requested
 *   path, budget, what); a matching line is applied without measuring, a new
 *   result is appended.  With DWG_TUNE_RELATIVE in what, w_budget is relative
 *   to the cloud's winding-number scale inside a closed surface, estimated
 *   from the geometry alone as mean(a) / (pi r^2 / 10), r the median distance
 *   to the 10th nearest other point over a sample of up to 2,048 points.
 *   On a batch handle every cloud is tuned on its own (the same what and
 *   budget; DWG_TUNE_RELATIVE is then the natural choice) and *out receives
 *   the settings of the largest cloud; the batch's one all-pairs launch keeps
 *   its fixed shapes, the per-cloud paths, leaf sizes, test forms and opening
 *   angles are the tuned ones.
 * dwg_get_tuning / dwg_set_tuning: read or apply settings (dwg_set_tuning
 *   fails with DWG_ERR_INVALID for a shape that is not compiled, a leaf size
 *   outside the list or theta outside (0, 1]; on a batch handle it applies to
 *   every cloud, and dwg_get_tuning reads the largest cloud's).  Settings change the order of floating-point additions, not
 *   the definition of the sums.
 */
#define DWG_TUNE_SHAPES 1
#define DWG_TUNE_TREE 2
#define DWG_TUNE_RELATIVE 4

typedef struct {
    int path;
    int points_pairs, points_threads;
    int corners_pairs, corners_threads;
    int tree_leaf;
    float theta;
    int tree_group;
    int knn_lists;
    double w_err;
    double ms_points, ms_corners;
    int from_cache;
} dwg_tuning;

int dwg_autotune(dwg_handle h, int what, double w_budget, const char *cache_path,
                 dwg_tuning *out);
int dwg_get_tuning(dwg_handle h, dwg_tuning *out);
int dwg_set_tuning(dwg_handle h, const dwg_tuning *t);

/*
 * The Barnes-Hut hierarchy the far field of Sec. 5.2 ("Octree Traversal")
 * walks, as built for the handle's current leaf size, opening angle and
 * regularisation, so that a caller can check it against the points.  The
 * hierarchy is a complete binary tree over leaves of `leaf` consecutive
 * points in Morton order: node 1 is the root, node k has children 2k and
 * 2k + 1, the nodes >= nodes / 2 are the leaves, and leaf b holds the sorted
 * points [b leaf, (b + 1) leaf) (empty past n).  Outputs (host or device;
 * each may be NULL except nodes_out and leaf_out):
 *   nodes_out   number of node slots (2 x the number of leaves; slot 0 unused),
 *   leaf_out    points per leaf,
 *   perm_out    int64 n: input index of each sorted point,
 *   area_out    double nodes: A = sum of the node's area weights,
 *   centre_out  double nodes x 3: area-weighted centre c,
 *   radius_out  double nodes: r, at least the largest
 *               distance of a node's point from c (exact for a leaf; for an
 *               inner node the largest |c_child - c| + r_child),
 *   record_out  float nodes x 4: the traversal record (c as float, the
 *               squared opening radius as float: (r / theta)^2, with the
 *               modified kernel max(r / theta, r + largest clamp radius)^2;
 *               -1 for an empty node).  A node is far for query q when
 *               |q - c|^2 > that value.
 * When cap < nodes only nodes_out and leaf_out are written.  Batch handles:
 * DWG_ERR_STATE.
 */
int dwg_get_tree(dwg_handle h, int64_t cap, int64_t *nodes_out, int *leaf_out, int64_t *perm_out,
                 double *area_out, double *centre_out, double *radius_out, float *record_out);

/*
 * k nearest input points (1 <= k <= 32) of m query points (float32 m x 3):
 * idx_out (int64 m x k, input-order indices, nearest first; ties in squared
 * float32 distance go to the smaller input index; -1 when n < k).
 */
int dwg_knn(dwg_handle h, const float *queries, int64_t m, int k, int64_t *idx_out);

/*
 * w at m query points for callers that cannot allocate device memory.
 * The paper has no counterpart: this is an engineering entry point.
 *
 * Who needs it: a caller that manages all device memory itself -- a
 * serving process with a fixed, pre-reserved HBM budget, a framework with its
 * own pool allocator -- or that cannot accept cudaMalloc/cudaFree inside its
 * work (cudaFree synchronises the whole device; an allocation may fail at any
 * point of a run).  This call performs no device allocation and calls no
 * allocating library routine.
 *
 * It computes the same w as dwg_eval_gwn with grad_out NULL (plain or
 * screened kernel, softened by eps, FP32 terms with compensated sums) for the
 * cloud given here, without a handle:
 *   points   float32 n x 3, normals float32 n x 3 (normalised here; zero
 *            vectors rejected), weights float32 n or NULL (a_i = 1),
 *   queries  float32 m x 3, w_out float32 m,
 * all in DEVICE memory of the current device (host pointers and pointers
 * into another GPU's memory are rejected with DWG_ERR_INVALID); the caller
 * sizes every array as stated (the library cannot check device lengths);
 * kernel, eps, screening as in dwg_set_params;
 * stream: the cudaStream_t to run on (NULL: the legacy default stream).
 * The call returns after w_out is written (it synchronises the stream).
 *
 * Limits: 1 <= n <= 65536 and 1 <= m <= 262144; larger sizes return
 * DWG_ERR_INVALID with a message naming the limit.  Its scratch (source
 * records, query records, partial sums, an error word: 15 MiB + 256 bytes)
 * is a fixed device array in the library, held by every GPU that loads the
 * library until the process exits.  The first call on a device looks up that
 * array's device address (cudaGetSymbolAddress, with that device current);
 * make that first call before any stream capture.  All calls share the one
 * array and it keeps the last call's contents: calls that overlap on the GPU
 * (other threads, other streams) race and must be serialised by the caller.
 * Errors are reported by the return code and dwg_last_error(NULL).
 */
int dwg_eval_w_noalloc(const float *points, const float *normals, const float *weights,
                       int64_t n, const float *queries, int64_t m, int kernel, float eps,
                       float screening, float *w_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DWG_H */
