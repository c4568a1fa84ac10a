// dwg_internal.cuh -- declarations shared by the CUDA translation units of
// libdwg.so: the engine context, device helpers and kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/dwg.h"

namespace dwg {

// ---------------------------------------------------------------------------
// constants
// ---------------------------------------------------------------------------
constexpr double kPi = 3.14159265358979323846;
constexpr int kMortonBits = 21;          // bits per axis of the point codes
constexpr int kMaxDepth = 14;            // octree depth cap
constexpr int kMaxK = 32;                // kNN cap
constexpr int kSrcFloats = 12;           // duplicated source record (x,x,y,y,z,z,mx,mx,...)
constexpr int kSrcFloatsClamp = 16;      // the same + (d2,d2,0,0), d2 = delta^2 (modified kernel)
constexpr int kSrcTile = 128;            // sources per shared-memory tile
constexpr int kBucket = 16;              // points per kNN bucket
constexpr int kSelBins = 4096;           // radix-select bins (level 1 and 2)
constexpr int kSearchBudget = 16384;     // node visits + distances of a face's own kNN search
constexpr int kDeferCap = 1 << 16;       // deferred faces per iteration (more: searched in place)
constexpr int kDeferBlocks = 256;        // blocks of the deferred-search launch

// device error flags (bitmask in ctx->d_err)
constexpr int kErrTimeout = 1;
constexpr int kErrNonfinite = 2;
constexpr int kErrOverflow = 4;
constexpr int kErrStack = 8;
constexpr int kErrGeometry = 16;  // a Voronoi cell outgrew its vertex buffer

// ---------------------------------------------------------------------------
// iteration state on the device (one struct, updated by kernels)
// ---------------------------------------------------------------------------
struct IterState {
    int iter;            // iterations performed in the current orient
    int done;            // converged flag
    int max_iters;
    int nfaces;          // faces emitted in the current iteration
    int ndefer;          // faces whose k-nearest search was deferred (kNN scatter)
    double iso;          // w_bar of the current iteration
    double stat;         // convergence statistic of the current iteration
};

#ifdef __CUDACC__
// a cloud whose loop has ended (converged, or at its iteration cap) skips
// the rest of a batched iteration
__device__ __forceinline__ bool cloud_idle(const IterState *st)
{
    return st->done || st->iter >= st->max_iters;
}

// Many clouds in one launch: blocks [off[c], off[c + 1]) of the grid run
// cloud c's blocks (clouds may have none).  Returns the cloud of this block.
__device__ __forceinline__ int seg_cloud(const int *__restrict__ off, int ncl)
{
    const int b = (int)blockIdx.x;
    int lo = 0, hi = ncl - 1;
    while (lo < hi) {  // the last cloud whose first block is <= b
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}
#endif

// radix-select state of the convergence statistic (device)
struct SelState {
    unsigned prefix;     // bits of the threshold found so far
    unsigned krem;       // rank still to find below the prefix
    unsigned above;      // values strictly above the threshold
    unsigned pad;
};

struct EvalParams {
    float eps2;        // eps^2
    float s;           // sqrt(lambda)
    float s2;          // lambda
    float nl2e_s;      // -sqrt(lambda) * log2(e)
    int screened;
};

// one cloud of a batched evaluation launch
struct GwnCloud {
    const float *src;
    int64_t ntiles;
    const float4 *q;
    int64_t m;
    int tpc;           // source tiles per chunk
    float *part;
    int64_t stride;
    EvalParams ep;
    const IterState *st;
};
struct GwnItem {
    int cloud, qtile, chunk, pad;
};

// the kNN bucket tree of a cloud as the device searches see it
struct KnnTree {
    const float4 *p4;
    const int64_t *perm;
    const uint64_t *codes;  // sorted 63-bit Morton codes of the points
    int64_t n;
    const float4 *lo, *hi;
    int levels;
    double cube_lo[3];
    double inv_h21;
};

// the root cube's quantisation (Morton codes of arbitrary queries)
struct CubeQ {
    double lo[3];
    double inv_h21;
};

// Everything one cloud's per-iteration kernels read, gathered for the
// batched launches of a batch handle: one entry per cloud in a device table,
// and per phase the offsets of each cloud's blocks in the launch's grid.
struct CloudIter {
    IterState *st;
    int *err;
    unsigned long long *counter;
    int64_t n;
    EvalParams ep;
    // reduce at the points (w and grad w, the iso-value's block sums)
    const float *part_p;
    int nchunks_p;
    const float4 *p4;
    const float *src;
    const uint64_t *codes;
    CubeQ cq;
    float4 *wg;
    double *wsum_blocks;
    int wsum_nb;
    // w at the corners
    const float *part_c;
    int nchunks_c;
    int64_t ncorners;
    float *wc;
    // level set
    const int *leaf_corners;
    const int4 *leaves;
    int64_t nleaves;
    const float4 *corner_pos;
    float4 *faces;
    int64_t max_faces;
    int2 *defer;
    int knn_budget;
    // kNN scatter
    KnnTree T;
    int k;
    const int64_t *cell_off;
    const int *cell_idx;
    double acc_scale;
    unsigned long long *acc;
    // normal update and convergence
    int mode;
    float4 *nrm;
    float *src_rw;
    float *dtheta;
    double *dn_blocks;
    struct SelState *sel;
    unsigned *sel_hist;
    double *sel_part;
    int sel_nb;
    float tol;
    int conv_rule;
    double *tr_iso, *tr_stat, *tr_dn;
    long long *tr_faces;
    // Barnes-Hut (tree clouds): moments and the two query sets' lists
    int tree;
    int levels, bucket;
    const float4 *nrm_c;
    double *tree_M;
    const float4 *tree_rec;
    float4 *tree_mrec, *tree_frec;
    const float4 *lq[2];          // [0] points, [1] corners
    int64_t lm[2];
    const int64_t *far_off[2], *near_off[2], *item_off[2];
    const int *far_ids[2], *near_ids[2];
    const int2 *items[2];
    int64_t nitems[2];
    float *ipart[2];
    float *lpart[2];              // the reduce's chunk-0 partials
};

// phases of a batched iteration (one launch each, every cloud's blocks)
enum BatchPhase {
    kPhReducePoints, kPhReduceW, kPhIso, kPhMcFaces, kPhKnn, kPhKnnDefer, kPhUpdate, kPhSelHist,
    kPhSelFind,
    kPhSelSum, kPhSelFinal, kPhLeafMom, kPhMomRec, kPhListsP, kPhListsC, kPhCombineP,
    kPhCombineC, kPhCount
};

// interaction lists of one query set for the group form of the Barnes-Hut
// test: per group of 64 queries the far node ids and the near leaf ids
struct TreeLists {
    const float4 *q = nullptr;       // the query array they were built for
    int64_t m = 0;
    uint64_t key = 0;                // tree generation, beta, depth they were built for
    int64_t *d_far_off = nullptr;    // ngroups + 1 offsets into d_far
    int64_t *d_near_off = nullptr;   // ngroups + 1 offsets into d_near
    int *d_far = nullptr, *d_near = nullptr;
    int64_t nfar = 0, nnear = 0;
    // work items: (group, first record) of at most a fixed number of
    // records each, their offsets per group and their partial sums
    int64_t *d_item_off = nullptr;
    int2 *d_items = nullptr;
    float *d_ipart = nullptr;
    int64_t nitems = 0;
    bool valid = false;
};

// ---------------------------------------------------------------------------
// engine context
// ---------------------------------------------------------------------------
struct Ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t own_stream = nullptr;
    std::string err;

    int64_t n = 0;        // points
    int64_t npad = 0;     // sources padded to a multiple of kSrcTile
    // parameters
    int kernel = DWG_KERNEL_PLAIN;
    float eps = 0.f, lambda = 0.f, tol = 0.1f;
    int conv_rule = DWG_CONV_TOP1;
    int max_iters = 30;
    int depth = 8, knn = 10, mode = DWG_UPDATE_LEVELSET;
    int init_mode = DWG_INIT_RANDOM;
    uint64_t seed = 1;
    bool normals_pending = true;   // initial normals must be (re)generated
    float *d_mlp_params = nullptr; // learned warm start (12,675 fp32 parameters)

    // geometry (sorted along the Morton curve)
    double cube_lo[3] = {0, 0, 0};
    double cube_L = 1.0;
    double bbox_c[3] = {0, 0, 0};  // bounding-box centre (Gauss-map initialisation)
    float4 *d_p4 = nullptr;        // (x, y, z, a) sorted
    int64_t *d_perm = nullptr;     // sorted index -> input index
    uint64_t *d_codes = nullptr;   // 63-bit Morton codes, sorted
    float *d_src = nullptr;        // npad x kSrcFloats source records
    // modified Poisson kernel (Sec. 5.2): rho = max(|p_j - q|, delta_j)
    int reg_mode = 0;              // DWG_REG_SOFTEN or DWG_REG_CLAMP
    bool compensated = true;       // two-sum fold of the all-pairs tile sums
    float *d_delta2 = nullptr;     // n: delta_j^2, sorted order
    float *d_src16 = nullptr;      // npad x kSrcFloatsClamp records (DWG_REG_CLAMP)
    float4 *d_nrm = nullptr;       // current normals, sorted
    float4 *d_nrm_init = nullptr;  // given initial normals, sorted
    float *d_dtheta = nullptr;
    float4 *d_wg = nullptr;        // (gx, gy, gz, w) at the points

    // kNN bucket hierarchy: complete binary tree over buckets of kBucket points
    int knn_levels = 0;            // leaves at level knn_levels (2^levels leaves)
    float4 *d_bvh_lo = nullptr;    // node AABB min (x,y,z,_)
    float4 *d_bvh_hi = nullptr;    // node AABB max

    // discretisation (depth-dependent)
    int built_depth = -1;
    int64_t nleaves = 0, ncorners = 0, max_faces = 0;
    int4 *d_leaves = nullptr;          // (level, code lo32, code hi32, nonempty) per leaf
    // per-leaf candidate lists of the faces' kNN (CSR over the leaves; a leaf
    // with an empty range keeps the tree search)
    int knn_lists = 1;
    int knn_budget = kSearchBudget;    // see dwg_set_knn_budget
    int64_t *d_cell_off = nullptr;     // nleaves + 1
    int *d_cell_idx = nullptr;         // sorted point indices
    int cells_k = 0;                   // k the lists were built for (0: none)
    int *d_leaf_corners = nullptr;     // nleaves x 8 corner indices
    uint64_t *d_corner_keys = nullptr; // Morton keys of corners (sorted)
    float4 *d_corner_pos = nullptr;
    float *d_wc = nullptr;             // w at corners
    float4 *d_faces = nullptr;         // 2 x max_faces: area vector, centroid
    int2 *d_defer = nullptr;           // kDeferCap deferred faces: (face, bound bits)
    unsigned long long *d_acc = nullptr; // n x 3 fixed-point face sums
    double acc_scale = 1.0;

    // evaluator shapes (indices into the variant tables of dwg_eval.cu) and
    // what the last autotune measured
    int var_grad = 0, var_w = 0;
    double tune_w_err = 0.0, tune_ms_points = 0.0, tune_ms_corners = 0.0;

    // evaluation scratch: partial sums per source chunk
    int nchunks_p = 1, nchunks_c = 1;
    float *d_part_p = nullptr;   // [nchunks][4][2][n]
    float *d_part_c = nullptr;   // [nchunks][2][ncorners]
    size_t part_p_cap = 0, part_c_cap = 0;
    double *d_wsum_blocks = nullptr;  // per-block w sums at the points
    int wsum_blocks = 0;
    double *d_dn_blocks = nullptr;    // per-block sums of |n_new - n_old|
    // convergence select: state, 4096 global bins, per-block partial sums
    SelState *d_sel = nullptr;
    unsigned *d_sel_hist = nullptr;
    double *d_sel_part = nullptr;

    // iteration state and traces
    IterState *d_state = nullptr;
    double *d_tr_iso = nullptr, *d_tr_stat = nullptr, *d_tr_dn = nullptr;
    long long *d_tr_faces = nullptr;
    int trace_cap = 0;
    int *d_err = nullptr;

    // Barnes-Hut far field over a binary tree of Morton ranges
    int path = DWG_PATH_AUTO;
    float tree_beta = 2.0f;            // 1 / opening angle
    int tree_leaf = 16;                // points per tree leaf (16, 32, 64 or 128)
    int tree_group = 1;                // 1: opening test per 64-query group, 0: per query
    int batch_phases = 1;              // batch handles: lanes of batched phases, 0 branches
    uint64_t tree_gen = 0;             // counts tree builds
    TreeLists lists_p, lists_c;        // group-test lists at the points and corners
    int tree_levels = 0;               // 2^tree_levels leaves
    bool tree_built = false;
    double tree_beta_set = -1.0;
    int tree_rec_dgen = -1;            // delta_gen the traversal records were built for
    int delta_gen = 0;                 // bumped whenever the clamp radii change
    double *d_tree_dmax = nullptr;     // largest clamp radius per node (modified kernel)
    double *d_tree_A = nullptr, *d_tree_C = nullptr, *d_tree_R = nullptr, *d_tree_M = nullptr;
    float4 *d_tree_rec = nullptr, *d_tree_mrec = nullptr;
    float4 *d_tree_frec = nullptr;     // node as a duplicated 48-byte source record
    unsigned long long *d_counter = nullptr;  // kernel evaluations of the tree path

    // graph; bufgen counts reallocations of buffers a captured graph refers
    // to, graph_gen is the count the graph was captured with
    cudaGraphExec_t graph_exec = nullptr;
    bool graph_valid = false;
    uint64_t bufgen = 0, graph_gen = ~0ull;

    // last results
    dwg_stats stats{};
    std::vector<double> tr_iso, tr_stat, tr_dn;
    std::vector<int64_t> tr_faces;
};

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
#define DWG_CUDA_TRY(ctx, call)                                                   \
    do {                                                                          \
        cudaError_t e_ = (call);                                                  \
        if (e_ != cudaSuccess) {                                                  \
            (ctx)->err = std::string(#call) + ": " + cudaGetErrorString(e_);      \
            return (e_ == cudaErrorMemoryAllocation) ? DWG_ERR_OOM : DWG_ERR_CUDA; \
        }                                                                         \
    } while (0)

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Morton interleave of a 21-bit value (bit k goes to bit 3k).
__host__ __device__ __forceinline__ uint64_t spread3(uint64_t v)
{
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}
// inverse of spread3
__host__ __device__ __forceinline__ uint64_t compact3(uint64_t v)
{
    v &= 0x1249249249249249ull;
    v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ull;
    v = (v ^ (v >> 4)) & 0x100f00f00f00f00full;
    v = (v ^ (v >> 8)) & 0x1f0000ff0000ffull;
    v = (v ^ (v >> 16)) & 0x1f00000000ffffull;
    v = (v ^ (v >> 32)) & 0x1fffffull;
    return v;
}
__host__ __device__ __forceinline__ uint64_t morton3(uint64_t x, uint64_t y, uint64_t z)
{
    return spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
}

#ifdef __CUDACC__
// Cell index along one axis at 2^21 cells per cube edge: floor((x - lo) * inv_h)
// clamped to [0, 2^21 - 1], with explicitly rounded double operations (no
// contraction) so that the result is reproducible bit for bit.
__device__ __forceinline__ int64_t quant21(float x, double lo, double inv_h)
{
    double t = __dmul_rn(__dsub_rn((double)x, lo), inv_h);
    double f = floor(t);
    if (f < 0.0) return 0;
    if (f > 2097151.0) return 2097151;
    return (int64_t)f;
}
#endif

// ---------------------------------------------------------------------------
// launchers (defined in the .cu files); all return cudaGetLastError()
// ---------------------------------------------------------------------------
// dwg_build.cu
// exclusive scan of n int64 values; *d_total (device) receives the sum
int scan_i64(Ctx *c, const int64_t *in, int64_t *out, int64_t n, int64_t *d_total);
cudaError_t launch_check_finite(const float *xyz, int64_t n, int *err, cudaStream_t s);
cudaError_t launch_bbox(const float *xyz, int64_t n, float *d_minmax /*6*/, cudaStream_t s);
cudaError_t launch_morton(const float *xyz, int64_t n, double lo0, double lo1, double lo2,
                          double inv_h21, uint64_t *keys, int64_t *idx, cudaStream_t s);
int radix_sort_pairs(Ctx *c, uint64_t *keys, int64_t *vals, int64_t n, int key_bits);
cudaError_t launch_gather_points(const float *xyz, const float *a, const int64_t *perm,
                                 int64_t n, float4 *p4, cudaStream_t s);
int build_knn_tree(Ctx *c);
int build_discretization(Ctx *c, int depth);

// dwg_eval.cu
EvalParams make_eval_params(const Ctx *c);
int eval_chunks(const Ctx *c, int64_t m, bool grad);
int eval_launch(Ctx *c, const float4 *q, int64_t m, bool grad, int nchunks, float *part,
                int64_t stride);
// evaluator shapes for the tuner: count, (P, NT) of variant v, chunking and
// launch of a given variant
int eval_variant_count(bool grad);
void eval_variant_shape(bool grad, int v, int *p, int *nt);
int eval_chunks_variant(const Ctx *c, int64_t m, bool grad, int v);
int eval_launch_variant(Ctx *c, const float4 *q, int64_t m, bool grad, int v, int nchunks,
                        float *part, int64_t stride);
cudaError_t launch_pack_sources(const float4 *p4, const float4 *nrm, int64_t n, int64_t npad,
                                float *src, cudaStream_t s);
cudaError_t launch_reduce_points(Ctx *c, const float *part, int nchunks, int64_t m,
                                 const float4 *queries, int self_mode, bool grad, float4 *out,
                                 double *wsum_blocks);
cudaError_t launch_reduce_w(Ctx *c, const float *part, int nchunks, int64_t m, float *out);
int batch_query_tile(bool grad);
cudaError_t launch_gwn_batch(const GwnCloud *clouds, const GwnItem *items, int64_t nitems,
                             bool grad, bool screened, int *err, cudaStream_t s);
int wsum_block_count(int64_t n);
int gwn_w_chunks_raw(int64_t m, int64_t npad, int device);
cudaError_t launch_gwn_w_raw(const float *src, int64_t npad, const float4 *q, int64_t m,
                             int nchunks, float *part, const EvalParams &ep, int *err,
                             cudaStream_t s);
cudaError_t launch_reduce_w_raw(const float *part, int nchunks, int64_t m, float *out,
                                cudaStream_t s);

// dwg_api.cu
void set_global_error(const std::string &msg);
bool use_tree(const Ctx *c);
// iteration buffers, spatial structures and source records of the current
// normals, as before an iteration
int engine_prepare(Ctx *c);

// dwg_tune.cu
void tuning_of(const Ctx *c, dwg_tuning *t);
int apply_tuning(Ctx *c, const dwg_tuning *t);
int autotune(Ctx *c, int what, double w_budget, const char *cache_path, dwg_tuning *out);

// dwg_tree.cu
void free_tree(Ctx *c);
int build_tree(Ctx *c);
int tree_records(Ctx *c);
cudaError_t launch_tree_moments(Ctx *c);
// st: loop state whose end makes the kernel skip its work (NULL: always run)
cudaError_t launch_tree_gwn(Ctx *c, const float4 *q, int64_t m, bool grad, float *part,
                            int64_t stride, const IterState *st);
// the interaction lists of a query set (group test); *built = false when the
// lists would not fit in device memory (the walk then runs every iteration)
int tree_lists(Ctx *c, TreeLists &L, const float4 *q, int64_t m, bool *built);
void free_lists(TreeLists &L);
// one iteration's tree evaluation of a query set: the cached lists when they
// are valid for it, else the walk
cudaError_t launch_tree_iter(Ctx *c, TreeLists &L, const float4 *q, int64_t m, bool grad,
                             float *part, int64_t stride, const IterState *st);

// batched iteration phases over a device table of CloudIter (one per cloud)
// and the block offsets `off` (ncl + 1) of the phase; `blocks` = off[ncl];
// `arg`: the select level (kPhSelHist, kPhSelFind) or the tree level
// (kPhLevelMom, see launch_tree_batch)
cudaError_t launch_iter_batch(int phase, const CloudIter *cl, const int *off, int ncl,
                              int blocks, int arg, cudaStream_t s);
cudaError_t launch_eval_batch(int phase, const CloudIter *cl, const int *off, int ncl,
                              int blocks, cudaStream_t s);
// kPhLeafMom, kPhMomRec, kPhListsP/C, kPhCombineP/C; level >= 0: the moments
// of tree level `level` (nodes [2^level, 2^(level + 1)) of every cloud)
cudaError_t launch_tree_batch(int phase, const CloudIter *cl, const int *off, int ncl,
                              int blocks, int level, bool screened, cudaStream_t s);
// blocks a cloud's part of a batched tree phase takes (0: none); level >= 0:
// the moments of that tree level
int tree_phase_blocks(const Ctx *c, int phase, int level);
bool tree_lists_current(const Ctx *c, bool corners);
void fill_cloud_iter(const Ctx *c, CloudIter *out);

// dwg_iter.cu
cudaError_t launch_iso(Ctx *c);
cudaError_t launch_mc_faces(Ctx *c);
cudaError_t launch_knn_scatter(Ctx *c);
cudaError_t launch_normal_update(Ctx *c);
cudaError_t launch_select(Ctx *c, cudaGraphConditionalHandle cond, int use_cond);
int select_blocks(int64_t n);
cudaError_t launch_random_normals(float4 *nrm, const int64_t *perm, int64_t n, uint64_t seed,
                                  cudaStream_t s);
cudaError_t launch_knn_query(Ctx *c, const float4 *q, int64_t m, int k, int64_t *idx_out);
// PCA (kPcaK nearest points) and Gauss-map initial normals over d_nrm
constexpr int kPcaK = 10;
cudaError_t launch_init_pca(Ctx *c);
cudaError_t launch_init_gauss(Ctx *c);
// local-Voronoi area weights of the m nearest points into p4.w (scratch: n + 1
// doubles; a_out: n floats in input order, device, or null)
cudaError_t launch_voronoi_weights(Ctx *c, int m, double *scratch, float *a_out);
// clamp radii of the modified kernel into d_delta2 (k in [1, 31]); delta_out:
// n floats in input order (device) or null
cudaError_t launch_clamp_delta(Ctx *c, int k, double vmin, double vmax, float *delta_out);
cudaError_t launch_pack_sources16(const Ctx *c);
// one CTA waiting on an mbarrier nothing arrives at, `polls` polls (the
// failure-detection self-check)
cudaError_t launch_wait_selfcheck(Ctx *c, int polls);
// measured FP32 issue rates of this device: packed-FMA lane operations and
// MUFU rsqrt per second
int measure_fp32_peaks(int device, double *ffma_lane_ops, double *rsqrt_ops, double *ex2_ops);
// the level set's triangles (count only with out null; counter: device)
cudaError_t launch_mc_tris(Ctx *c, float *out, int64_t cap, unsigned long long *counter);
// per-leaf candidate lists for the faces' k nearest points (once per
// discretisation and k; skipped when they would not fit comfortably)
int build_cell_lists(Ctx *c);
void free_cell_lists(Ctx *c);
// distance to the 10th nearest other point for m points sampled evenly
cudaError_t launch_spacing(Ctx *c, int64_t m, float *d_out);
cudaError_t launch_features(Ctx *c, float *X, bool by_input, double *cR);
cudaError_t launch_normals_from_y(Ctx *c, const float *Y);

// dwg_mlp.cu
constexpr int kMlpParamCount = 12675;
// err: device flag for a wait that gave up (NULL: the library's own flag,
// read and cleared by mlp_forward_error)
cudaError_t launch_mlp_forward(const float *P, const float *X, int64_t B, float *Y, cudaStream_t s,
                               int *err);
int mlp_forward_error(cudaStream_t s);
cudaError_t launch_mlp_grad(const float *P, const float *X, const float *T, int64_t B, float *grad,
                            double *loss, cudaStream_t s);
cudaError_t launch_adam(float *p, const float *g, float *m, float *v, int step, float lr,
                        cudaStream_t s);

}  // namespace dwg
