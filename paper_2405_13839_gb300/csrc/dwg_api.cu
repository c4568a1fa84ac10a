// dwg_api.cu -- the C ABI (include/dwg.h) and the host engine around the
// kernels: handle state, pointer classification, buffer management, the
// iteration body of Alg. 1 and its capture into a CUDA graph whose
// conditional WHILE node repeats the body until the convergence rule of
// Sec. 5.1 holds (no host synchronisation between iterations).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "dwg_internal.cuh"


using namespace dwg;

struct dwg_ctx : public Ctx {
    // batch handles (dwg_create_batch): one sub-handle per cloud
    bool is_batch = false;
    std::vector<dwg_ctx *> clouds;
    std::vector<int64_t> offsets;
    GwnCloud *d_bcl_p = nullptr, *d_bcl_c = nullptr;
    GwnItem *d_bit_p = nullptr, *d_bit_c = nullptr;
    int64_t nit_p = 0, nit_c = 0;
    IterState **d_states = nullptr;
    bool eps_given = false;
    // fork / join of the clouds' chains in a batch iteration (each cloud runs
    // on its own stream, so the graph holds one branch per cloud)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // batched phases: the clouds are split over a few lanes (streams); in
    // each lane every phase is one launch over the lane's clouds.  The
    // clouds' argument table (lane by lane) and, per lane, phase and tree
    // level, the offsets of each cloud's blocks in the phase's grid.
    struct Lane {
        std::vector<dwg_ctx *> clouds;
        int base = 0;                  // first entry of the lane in d_citer
        size_t off_base = 0;           // first offset of the lane in d_boff
        int ph_blocks[kPhCount] = {};
        std::vector<int> lv_blocks;    // per tree level
        std::vector<dwg_ctx *> walk_p, walk_c;  // tree clouds without current lists
    };
    std::vector<Lane> lanes;
    CloudIter *d_citer = nullptr;
    int *d_boff = nullptr;
    bool batched = false;              // the batched phases apply (uniform settings)
};

static std::mutex g_err_mu;
static std::string g_create_err;

namespace dwg {
// last error of the calls that have no handle (reported by dwg_last_error(NULL))
void set_global_error(const std::string &msg)
{
    std::lock_guard<std::mutex> lk(g_err_mu);
    g_create_err = msg;
}
}  // namespace dwg

namespace dwg {
bool use_tree(const Ctx *c)
{
    if (c->path == DWG_PATH_TREE) return true;
    if (c->path == DWG_PATH_ALLPAIRS) return false;
    return c->n > 65536;
}
}  // namespace dwg

static int fail(Ctx *c, int code, const std::string &msg)
{
    if (c) c->err = msg;
    return code;
}

// Memory that the library's kernels may read or write directly: device
// memory of the current device, or managed memory.  A pointer into another
// GPU's memory is not (without peer access a kernel could not touch it); such
// buffers, like host memory, are staged with cudaMemcpy.
static bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

// Memory the host may read with memcpy (pageable or page-locked host memory).
static bool is_host_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return a.type == cudaMemoryTypeUnregistered || a.type == cudaMemoryTypeHost;
}

// Copy bytes between a caller buffer (host memory, or device memory of any
// GPU) and the handle's device memory; the unified address space tells the
// copy which kind it is.
static int upload(Ctx *c, void *dst, const void *src, size_t bytes)
{
    DWG_CUDA_TRY(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c->stream));
    return DWG_OK;
}
static int download(Ctx *c, void *dst, const void *src, size_t bytes)
{
    DWG_CUDA_TRY(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c->stream));
    return DWG_OK;
}

// ---------------------------------------------------------------------------
// small kernels used only by the engine
// ---------------------------------------------------------------------------
// normals: caller layout (input order, float xyz) -> sorted float4, normalised
__global__ void k_normals_in(const float *__restrict__ v, const int64_t *__restrict__ perm,
                             int64_t n, float4 *out, int *err)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t j = perm[i];
    float x = v[3 * j], y = v[3 * j + 1], z = v[3 * j + 2];
    float l = sqrtf(x * x + y * y + z * z);
    if (!(l > 0.f) || !isfinite(l)) {
        atomicOr(err, kErrNonfinite);
        l = 1.f;
    }
    // a vector of unit length to float rounding is taken as is, so that
    // normals read back from the library resume an orientation bit for bit
    if (fabsf(l - 1.f) <= 4e-7f) l = 1.f;
    out[i] = make_float4(x / l, y / l, z / l, 0.f);
}
// sorted float4 -> caller layout (input order)
__global__ void k_normals_out(const float4 *__restrict__ v, const int64_t *__restrict__ perm,
                              int64_t n, float *out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t j = perm[i];
    float4 a = v[i];
    out[3 * j] = a.x;
    out[3 * j + 1] = a.y;
    out[3 * j + 2] = a.z;
}
__global__ void k_scalar_out(const float *__restrict__ v, const int64_t *__restrict__ perm,
                             int64_t n, float *out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[perm[i]] = v[i];
}
__global__ void k_wg_out(const float4 *__restrict__ v, const int64_t *__restrict__ perm, int64_t n,
                         float *w, float *g)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t j = perm ? perm[i] : i;
    float4 a = v[i];
    if (w) w[j] = a.w;
    if (g) {
        g[3 * j] = a.x;
        g[3 * j + 1] = a.y;
        g[3 * j + 2] = a.z;
    }
}
__global__ void k_xyz_to_f4(const float *__restrict__ v, int64_t m, float4 *out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) out[i] = make_float4(v[3 * i], v[3 * i + 1], v[3 * i + 2], 0.f);
}
__global__ void k_weights_in(const float *__restrict__ a, const int64_t *__restrict__ perm,
                             int64_t n, float4 *p4, int *err)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float v = a[perm[i]];
    if (!(v > 0.f) || !isfinite(v)) atomicOr(err, kErrNonfinite);
    p4[i].w = v;
}
__global__ void k_iter_reset(IterState *st, int max_iters, unsigned long long *counter)
{
    if (counter) *counter = 0ull;
    st->iter = 0;
    st->done = 0;
    st->max_iters = max_iters;
    st->nfaces = 0;
    st->ndefer = 0;
    st->iso = 0.0;
    st->stat = 0.0;
}

#define LAUNCH_CHECK(c)                                                                  \
    do {                                                                                 \
        cudaError_t e_ = cudaGetLastError();                                             \
        if (e_ != cudaSuccess) return fail(c, DWG_ERR_CUDA, cudaGetErrorString(e_));     \
    } while (0)

static unsigned nblk(int64_t n, int b = 256) { return (unsigned)ceil_div(n, b); }

// ---------------------------------------------------------------------------
// buffers
// ---------------------------------------------------------------------------
// octree of the handle's depth, its corners and their partial sums
static int ensure_levelset_buffers(Ctx *c, bool tree)
{
    if (c->built_depth != c->depth) ++c->bufgen;
    int rc = build_discretization(c, c->depth);
    if (rc) return rc;
    const int nch_c = tree ? 1 : eval_chunks(c, c->ncorners, false);
    if (nch_c != c->nchunks_c) ++c->bufgen;
    c->nchunks_c = nch_c;
    size_t need_c = (size_t)c->nchunks_c * 2 * (size_t)c->ncorners;
    if (need_c > c->part_c_cap) {
        cudaFree(c->d_part_c);
        c->d_part_c = nullptr;
        ++c->bufgen;
        DWG_CUDA_TRY(c, cudaMalloc(&c->d_part_c, need_c * sizeof(float)));
        c->part_c_cap = need_c;
    }
    return DWG_OK;
}

static int ensure_iter_buffers(Ctx *c)
{
    const bool tree = use_tree(c);
    if (tree) {
        int rc = build_tree(c);
        if (!rc) rc = tree_records(c);
        if (rc) return rc;
    }
    // partial sums for the point evaluation
    const int nch_p = tree ? 1 : eval_chunks(c, c->n, true);
    if (nch_p != c->nchunks_p) ++c->bufgen;
    c->nchunks_p = nch_p;
    size_t need_p = (size_t)c->nchunks_p * 8 * (size_t)c->n;
    if (need_p > c->part_p_cap) {
        cudaFree(c->d_part_p);
        c->d_part_p = nullptr;
        ++c->bufgen;
        DWG_CUDA_TRY(c, cudaMalloc(&c->d_part_p, need_p * sizeof(float)));
        c->part_p_cap = need_p;
    }
    if (c->mode == DWG_UPDATE_LEVELSET) {
        int rc = ensure_levelset_buffers(c, tree);
        if (!rc) rc = build_cell_lists(c);
        if (rc) return rc;
    }
    // group form of the Barnes-Hut test: interaction lists, built once
    if (tree && c->tree_group) {
        bool built = false;
        int rc = tree_lists(c, c->lists_p, c->d_p4, c->n, &built);
        if (!rc && c->mode == DWG_UPDATE_LEVELSET)
            rc = tree_lists(c, c->lists_c, c->d_corner_pos, c->ncorners, &built);
        if (rc) return rc;
    }
    if (c->trace_cap < c->max_iters) {
        ++c->bufgen;
        cudaFree(c->d_tr_iso);
        cudaFree(c->d_tr_stat);
        cudaFree(c->d_tr_dn);
        cudaFree(c->d_tr_faces);
        c->d_tr_iso = c->d_tr_stat = c->d_tr_dn = nullptr;
        c->d_tr_faces = nullptr;
        c->trace_cap = 0;
        DWG_CUDA_TRY(c, cudaMalloc(&c->d_tr_iso, c->max_iters * sizeof(double)));
        DWG_CUDA_TRY(c, cudaMalloc(&c->d_tr_stat, c->max_iters * sizeof(double)));
        DWG_CUDA_TRY(c, cudaMalloc(&c->d_tr_dn, c->max_iters * sizeof(double)));
        DWG_CUDA_TRY(c, cudaMalloc(&c->d_tr_faces, c->max_iters * sizeof(long long)));
        c->trace_cap = c->max_iters;
    }
    return DWG_OK;
}

static void invalidate_graph(Ctx *c)
{
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    c->graph_exec = nullptr;
    c->graph_valid = false;
}

// ---------------------------------------------------------------------------
// the iteration body (Alg. 1, one pass of the repeat loop)
// ---------------------------------------------------------------------------
// ev (optional): 10 events recorded around the body's launches for profiling
// snap (optional, device, 2 entries): the evaluation counter after the
// point and after the corner evaluation (profiling of the tree path)
static int enqueue_body(Ctx *c, cudaGraphConditionalHandle cond, int use_cond,
                        cudaEvent_t *ev = nullptr, unsigned long long *snap = nullptr)
{
    int rc;
    auto mark = [&](int k) {
        if (ev) cudaEventRecord(ev[k], c->stream);
    };
    const bool tree = use_tree(c);
    // w and grad w at the input points
    mark(0);
    if (tree) {
        if (launch_tree_moments(c) != cudaSuccess ||
            launch_tree_iter(c, c->lists_p, c->d_p4, c->n, true, c->d_part_p, c->n, c->d_state) !=
                cudaSuccess)
            return fail(c, DWG_ERR_CUDA, "tree launch failed");
    } else if ((rc = eval_launch(c, c->d_p4, c->n, true, c->nchunks_p, c->d_part_p, c->n))) {
        return rc;
    }
    mark(1);
    if (snap)
        cudaMemcpyAsync(snap, c->d_counter, sizeof(unsigned long long), cudaMemcpyDeviceToDevice,
                        c->stream);
    if (launch_reduce_points(c, c->d_part_p, c->nchunks_p, c->n, c->d_p4, 1, true, c->d_wg,
                             c->d_wsum_blocks) != cudaSuccess)
        return fail(c, DWG_ERR_CUDA, "reduce launch failed");
    mark(2);
    if (launch_iso(c) != cudaSuccess) return fail(c, DWG_ERR_CUDA, "iso launch failed");
    mark(3);
    if (c->mode == DWG_UPDATE_LEVELSET) {
        // w at the octree leaf corners, level set, face gradients to the k nearest points
        if (tree) {
            if (launch_tree_iter(c, c->lists_c, c->d_corner_pos, c->ncorners, false, c->d_part_c,
                                 c->ncorners, c->d_state) != cudaSuccess)
                return fail(c, DWG_ERR_CUDA, "tree launch failed");
        } else if ((rc = eval_launch(c, c->d_corner_pos, c->ncorners, false, c->nchunks_c,
                                     c->d_part_c, c->ncorners))) {
            return rc;
        }
        mark(4);
        if (snap)
            cudaMemcpyAsync(snap + 1, c->d_counter, sizeof(unsigned long long),
                            cudaMemcpyDeviceToDevice, c->stream);
        if (launch_reduce_w(c, c->d_part_c, c->nchunks_c, c->ncorners, c->d_wc) != cudaSuccess)
            return fail(c, DWG_ERR_CUDA, "reduce_w launch failed");
        mark(5);
        if (launch_mc_faces(c) != cudaSuccess) return fail(c, DWG_ERR_CUDA, "mc launch failed");
        mark(6);
        if (launch_knn_scatter(c) != cudaSuccess)
            return fail(c, DWG_ERR_CUDA, "knn launch failed");
        mark(7);
    } else {
        mark(4); mark(5); mark(6); mark(7);
    }
    if (launch_normal_update(c) != cudaSuccess) return fail(c, DWG_ERR_CUDA, "update launch failed");
    mark(8);
    if (launch_select(c, cond, use_cond) != cudaSuccess)
        return fail(c, DWG_ERR_CUDA, "select launch failed");
    mark(9);
    return DWG_OK;
}

// kernel launches in a captured graph (the iteration body)
static int count_kernel_nodes(cudaGraph_t g)
{
    size_t num = 0;
    if (cudaGraphGetNodes(g, nullptr, &num) != cudaSuccess || num == 0) return 0;
    std::vector<cudaGraphNode_t> nodes(num);
    if (cudaGraphGetNodes(g, nodes.data(), &num) != cudaSuccess) return 0;
    int k = 0;
    for (size_t i = 0; i < num; ++i) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
    }
    return k;
}

static int build_graph(Ctx *c)
{
    invalidate_graph(c);
    cudaGraph_t g = nullptr;
    DWG_CUDA_TRY(c, cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle cond;
    cudaError_t e = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return fail(c, DWG_ERR_CUDA, std::string("conditional handle: ") + cudaGetErrorString(e));
    }
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return fail(c, DWG_ERR_CUDA, std::string("conditional node: ") + cudaGetErrorString(e));
    }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    // capture on the library's own stream (never the legacy default stream)
    cudaStream_t saved = c->stream;
    c->stream = c->own_stream;
    e = cudaStreamBeginCaptureToGraph(c->stream, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
        c->stream = saved;
        cudaGraphDestroy(g);
        return fail(c, DWG_ERR_CUDA, std::string("begin capture: ") + cudaGetErrorString(e));
    }
    int rc = enqueue_body(c, cond, 1);
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(c->stream, &captured);
    c->stream = saved;
    if (rc || e != cudaSuccess) {
        cudaGraphDestroy(g);
        if (rc) return rc;
        return fail(c, DWG_ERR_CUDA, std::string("end capture: ") + cudaGetErrorString(e));
    }
    c->stats.kernels_per_iteration = count_kernel_nodes(body);
    e = cudaGraphInstantiate(&c->graph_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->graph_exec = nullptr;
        return fail(c, DWG_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e));
    }
    c->graph_valid = true;
    c->graph_gen = c->bufgen;
    return DWG_OK;
}

static int check_device_err(Ctx *c)
{
    int herr = 0;
    DWG_CUDA_TRY(c, cudaMemcpyAsync(&herr, c->d_err, sizeof(int), cudaMemcpyDeviceToHost,
                                    c->stream));
    DWG_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (herr) {
        DWG_CUDA_TRY(c, cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
        if (herr & kErrTimeout) return fail(c, DWG_ERR_TIMEOUT, "a device-side wait gave up");
        if (herr & kErrNonfinite) return fail(c, DWG_ERR_NONFINITE, "non-finite or invalid input");
        if (herr & kErrOverflow) return fail(c, DWG_ERR_CUDA, "face buffer overflow");
        if (herr & kErrStack) return fail(c, DWG_ERR_CUDA, "kNN traversal stack overflow");
        if (herr & kErrGeometry) return fail(c, DWG_ERR_CUDA, "Voronoi cell vertex overflow");
        return fail(c, DWG_ERR_CUDA, "device error flag set");
    }
    return DWG_OK;
}

// initial normals into d_nrm and source records from them
static int prepare_normals(Ctx *c)
{
    if (c->normals_pending) {
        if (c->init_mode != DWG_INIT_GIVEN) {
            // the random draw is also the fallback of the other modes
            if (launch_random_normals(c->d_nrm, c->d_perm, c->n, c->seed, c->stream) !=
                cudaSuccess)
                return fail(c, DWG_ERR_CUDA, "random normals launch failed");
            if (c->init_mode == DWG_INIT_PCA && launch_init_pca(c) != cudaSuccess)
                return fail(c, DWG_ERR_CUDA, "PCA normals launch failed");
            if (c->init_mode == DWG_INIT_GAUSS && launch_init_gauss(c) != cudaSuccess)
                return fail(c, DWG_ERR_CUDA, "Gauss-map normals launch failed");
            if (c->init_mode == DWG_INIT_LEARNED) {
                float *X = nullptr, *Y = nullptr;
                double *cR = nullptr;
                auto run = [&]() -> int {
                    DWG_CUDA_TRY(c, cudaMalloc(&X, c->n * 64 * sizeof(float)));
                    DWG_CUDA_TRY(c, cudaMalloc(&Y, c->n * 3 * sizeof(float)));
                    DWG_CUDA_TRY(c, cudaMalloc(&cR, 4 * sizeof(double)));
                    if (launch_features(c, X, false, cR) != cudaSuccess ||
                        launch_mlp_forward(c->d_mlp_params, X, c->n, Y, c->stream, c->d_err) !=
                            cudaSuccess ||
                        launch_normals_from_y(c, Y) != cudaSuccess)
                        return fail(c, DWG_ERR_CUDA, "learned init launch failed");
                    DWG_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
                    return DWG_OK;
                };
                int rc = run();
                cudaFree(X);
                cudaFree(Y);
                cudaFree(cR);
                if (rc) return rc;
            }
        } else {
            DWG_CUDA_TRY(c, cudaMemcpyAsync(c->d_nrm, c->d_nrm_init, c->n * sizeof(float4),
                                            cudaMemcpyDeviceToDevice, c->stream));
        }
        c->normals_pending = false;
    }
    if (launch_pack_sources(c->d_p4, c->d_nrm, c->n, c->npad, c->d_src, c->stream) != cudaSuccess)
        return fail(c, DWG_ERR_CUDA, "pack launch failed");
    if (c->reg_mode == DWG_REG_CLAMP && launch_pack_sources16(c) != cudaSuccess)
        return fail(c, DWG_ERR_CUDA, "pack launch failed");
    return DWG_OK;
}

namespace dwg {
int engine_prepare(Ctx *c)
{
    int rc = ensure_iter_buffers(c);
    if (!rc) rc = prepare_normals(c);
    return rc;
}
}  // namespace dwg

static double interactions_per_iter(const Ctx *c)
{
    // (the tree path counts its evaluations on the device instead)
    double n = (double)c->n;
    double it = n * n;
    if (c->mode == DWG_UPDATE_LEVELSET) it += (double)c->ncorners * n;
    return it;
}

// ---------------------------------------------------------------------------
// ABI
// ---------------------------------------------------------------------------
extern "C" {

const char *dwg_last_error(dwg_handle h)
{
    if (h) return h->err.c_str();
    std::lock_guard<std::mutex> lk(g_err_mu);
    return g_create_err.c_str();
}

void dwg_destroy(dwg_handle h)
{
    if (!h) return;
    for (dwg_ctx *c : h->clouds) dwg_destroy(c);
    h->clouds.clear();
    cudaFree(h->d_bcl_p);
    cudaFree(h->d_bcl_c);
    cudaFree(h->d_bit_p);
    cudaFree(h->d_bit_c);
    cudaFree(h->d_states);
    cudaFree(h->d_citer);
    cudaFree(h->d_boff);
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    invalidate_graph(h);
    void *bufs[] = {h->d_p4, h->d_perm, h->d_codes, h->d_src, h->d_nrm, h->d_nrm_init,
                    h->d_dtheta, h->d_wg, h->d_bvh_lo, h->d_bvh_hi, h->d_leaves,
                    h->d_leaf_corners, h->d_corner_keys, h->d_corner_pos, h->d_wc, h->d_faces,
                    h->d_acc, h->d_part_p, h->d_part_c, h->d_wsum_blocks, h->d_dn_blocks,
                    h->d_sel, h->d_sel_hist, h->d_sel_part,
                    h->d_state, h->d_tr_iso, h->d_tr_stat, h->d_tr_dn, h->d_tr_faces, h->d_err,
                    h->d_tree_A, h->d_tree_C, h->d_tree_R, h->d_tree_M, h->d_tree_rec,
                    h->d_tree_mrec, h->d_tree_frec, h->d_counter, h->d_mlp_params,
                    h->d_delta2, h->d_src16, h->d_cell_off, h->d_cell_idx, h->d_tree_dmax};
    for (void *p : bufs) cudaFree(p);
    free_lists(h->lists_p);
    free_lists(h->lists_c);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->own_stream) cudaStreamDestroy(h->own_stream);
    delete h;
}

static int create_impl(dwg_ctx *c, const float *points, int64_t n)
{
    DWG_CUDA_TRY(c, cudaGetDevice(&c->device));
    DWG_CUDA_TRY(c, cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking));
    c->stream = c->own_stream;
    c->n = n;
    c->npad = ceil_div(n, kSrcTile) * kSrcTile;
    DWG_CUDA_TRY(c, cudaMalloc(&c->d_err, sizeof(int)));
    DWG_CUDA_TRY(c, cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
    float *xyz = nullptr;
    bool own_xyz = false;
    if (is_device_ptr(points)) {
        xyz = const_cast<float *>(points);
    } else {
        DWG_CUDA_TRY(c, cudaMalloc(&xyz, n * 3 * sizeof(float)));
        own_xyz = true;
        int rc = upload(c, xyz, points, n * 3 * sizeof(float));
        if (rc) { cudaFree(xyz); return rc; }
    }
    auto body = [&]() -> int {
        if (launch_check_finite(xyz, 3 * n, c->d_err, c->stream) != cudaSuccess)
            return fail(c, DWG_ERR_CUDA, "finite-check launch failed");
        int rc = check_device_err(c);
        if (rc) return rc;
        float *mm = nullptr;
        DWG_CUDA_TRY(c, cudaMalloc(&mm, 6 * sizeof(float)));
        launch_bbox(xyz, n, mm, c->stream);
        float hm[6];
        DWG_CUDA_TRY(c, cudaMemcpyAsync(hm, mm, sizeof(hm), cudaMemcpyDeviceToHost, c->stream));
        DWG_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        cudaFree(mm);
        // root cube of the octree: bounding-box centre, edge 1.125 x largest extent
        double mn[3] = {hm[0], hm[1], hm[2]}, mx[3] = {hm[3], hm[4], hm[5]};
        double ext = 0.0;
        for (int k = 0; k < 3; ++k) ext = std::max(ext, mx[k] - mn[k]);
        double L = ext > 0.0 ? ext * 1.125 : 1.0;
        for (int k = 0; k < 3; ++k) {
            double cen = (mn[k] + mx[k]) * 0.5;
            c->bbox_c[k] = cen;
            c->cube_lo[k] = cen - L * 0.5;
        }
        c->cube_L = L;
        // default softening: half the spacing of n points over an extent^2 patch
        c->eps = (float)(0.5 * (ext > 0.0 ? ext : 1.0) / sqrt((double)n));
        // Morton order
        DWG_CUDA_TRY(c, cudaMalloc(&c->d_codes, n * sizeof(uint64_t)));
        DWG_CUDA_TRY(c, cudaMalloc(&c->d_perm, n * sizeof(int64_t)));
        double inv_h21 = (double)(1 << kMortonBits) / L;
        if (launch_morton(xyz, n, c->cube_lo[0], c->cube_lo[1], c->cube_lo[2], inv_h21,
                          c->d_codes, c->d_perm, c->stream) != cudaSuccess)
            return fail(c, DWG_ERR_CUDA, "morton launch failed");
        if ((rc = radix_sort_pairs(c, c->d_codes, c->d_perm, n, 3 * kMortonBits))) return rc;
        DWG_CUDA_TRY(c, cudaMalloc(&c->d_p4, n * sizeof(float4)));
        if (launch_gather_points(xyz, nullptr, c->d_perm, n, c->d_p4, c->stream) != cudaSuccess)
            return fail(c, DWG_ERR_CUDA, "gather launch failed");
        if ((rc = build_knn_tree(c))) return rc;
        // per-point buffers
        DWG_CUDA_TRY(c, cudaMalloc(&c->d_src, c->npad * kSrcFloats * sizeof(float)));
        DWG_CUDA_TRY(c, cudaMalloc(&c->d_nrm, n * sizeof(float4)));
        DWG_CUDA_TRY(c, cudaMalloc(&c->d_nrm_init, n * sizeof(float4)));
        DWG_CUDA_TRY(c, cudaMalloc(&c->d_dtheta, n * sizeof(float)));
        DWG_CUDA_TRY(c, cudaMalloc(&c->d_wg, n * sizeof(float4)));
        DWG_CUDA_TRY(c, cudaMalloc(&c->d_acc, 3 * n * sizeof(unsigned long long)));
        DWG_CUDA_TRY(c, cudaMemsetAsync(c->d_acc, 0, 3 * n * sizeof(unsigned long long), c->stream));
        c->wsum_blocks = wsum_block_count(n);
        DWG_CUDA_TRY(c, cudaMalloc(&c->d_wsum_blocks, c->wsum_blocks * sizeof(double)));
        DWG_CUDA_TRY(c, cudaMalloc(&c->d_dn_blocks, ceil_div(n, 256) * sizeof(double)));
        DWG_CUDA_TRY(c, cudaMalloc(&c->d_sel, sizeof(SelState)));
        DWG_CUDA_TRY(c, cudaMalloc(&c->d_sel_hist, kSelBins * sizeof(unsigned)));
        DWG_CUDA_TRY(c, cudaMemsetAsync(c->d_sel_hist, 0, kSelBins * sizeof(unsigned), c->stream));
        DWG_CUDA_TRY(c, cudaMalloc(&c->d_sel_part, select_blocks(n) * sizeof(double)));
        DWG_CUDA_TRY(c, cudaMalloc(&c->d_state, sizeof(IterState)));
        DWG_CUDA_TRY(c, cudaMalloc(&c->d_counter, sizeof(unsigned long long)));
        k_iter_reset<<<1, 1, 0, c->stream>>>(c->d_state, c->max_iters, nullptr);
        DWG_CUDA_TRY(c, cudaMemsetAsync(c->d_counter, 0, sizeof(unsigned long long), c->stream));
        DWG_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        c->stats.n_points = n;
        return DWG_OK;
    };
    int rc = body();
    if (own_xyz) {
        cudaStreamSynchronize(c->stream);
        cudaFree(xyz);
    }
    return rc;
}

int dwg_create(const float *points, int64_t n, dwg_handle *out)
{
    if (out) *out = nullptr;
    auto set_err = [](const std::string &m) {
        std::lock_guard<std::mutex> lk(g_err_mu);
        g_create_err = m;
    };
    if (!out || !points) {
        set_err("dwg_create: null argument");
        return DWG_ERR_INVALID;
    }
    if (n < 1 || n > ((int64_t)1 << 31) - 1) {
        set_err("dwg_create: n must be in [1, 2^31 - 1]");
        return DWG_ERR_INVALID;
    }
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        set_err(std::string("dwg_create: no usable CUDA device: ") + cudaGetErrorString(e));
        return DWG_ERR_CUDA;
    }
    dwg_ctx *c = new (std::nothrow) dwg_ctx();
    if (!c) {
        set_err("dwg_create: out of host memory");
        return DWG_ERR_OOM;
    }
    int rc = create_impl(c, points, n);
    if (rc) {
        set_err("dwg_create: " + c->err);
        dwg_destroy(c);
        return rc;
    }
    *out = c;
    return DWG_OK;
}

int dwg_set_stream(dwg_handle h, void *stream)
{
    if (!h) return DWG_ERR_INVALID;
    cudaStreamSynchronize(h->stream);
    h->stream = stream ? (cudaStream_t)stream : h->own_stream;
    return DWG_OK;
}

int dwg_set_params(dwg_handle h, int kernel, float eps, float screening, int max_iters, float tol)
{
    if (!h) return DWG_ERR_INVALID;
    if (kernel != DWG_KERNEL_PLAIN && kernel != DWG_KERNEL_SCREENED)
        return fail(h, DWG_ERR_INVALID, "kernel must be DWG_KERNEL_PLAIN or DWG_KERNEL_SCREENED");
    const bool keep_eps = h->is_batch && eps == 0.f;  // each cloud keeps its own softening
    if (!keep_eps && (!(eps > 0.f) || !isfinite(eps)))
        return fail(h, DWG_ERR_INVALID, "eps must be > 0 (0 on a batch handle: per-cloud default)");
    if (!(screening >= 0.f) || !isfinite(screening))
        return fail(h, DWG_ERR_INVALID, "screening must be >= 0");
    if (max_iters < 1 || max_iters > 100000)
        return fail(h, DWG_ERR_INVALID, "max_iters must be in [1, 100000]");
    if (!(tol > 0.f) || !isfinite(tol)) return fail(h, DWG_ERR_INVALID, "tol must be > 0");
    h->kernel = kernel;
    h->eps = eps;
    h->lambda = screening;
    h->max_iters = max_iters;
    h->tol = tol;
    h->eps_given = !keep_eps;
    invalidate_graph(h);
    for (dwg_ctx *c : h->clouds)
        dwg_set_params(c, kernel, keep_eps ? c->eps : eps, screening, max_iters, tol);
    return DWG_OK;
}

int dwg_set_convergence(dwg_handle h, int rule)
{
    if (!h) return DWG_ERR_INVALID;
    if (rule != DWG_CONV_TOP1 && rule != DWG_CONV_MEAN)
        return fail(h, DWG_ERR_INVALID, "rule must be DWG_CONV_TOP1 or DWG_CONV_MEAN");
    h->conv_rule = rule;
    invalidate_graph(h);
    for (dwg_ctx *c : h->clouds) dwg_set_convergence(c, rule);
    return DWG_OK;
}

int dwg_set_knn_budget(dwg_handle h, int budget)
{
    if (!h) return DWG_ERR_INVALID;
    if (budget < -1) return fail(h, DWG_ERR_INVALID, "budget must be >= -1");
    if (h->knn_budget != budget) {
        h->knn_budget = budget;
        invalidate_graph(h);
    }
    for (dwg_ctx *c : h->clouds) dwg_set_knn_budget(c, budget);
    return DWG_OK;
}

int dwg_set_batch_mode(dwg_handle h, int lanes)
{
    if (!h) return DWG_ERR_INVALID;
    if (!h->is_batch) return fail(h, DWG_ERR_STATE, "dwg_set_batch_mode needs a batch handle");
    if (lanes < 0 || lanes > DWG_MAX_BATCH_LANES)
        return fail(h, DWG_ERR_INVALID, "lanes must be in [0, DWG_MAX_BATCH_LANES]");
    if (h->batch_phases != lanes) {
        h->batch_phases = lanes;
        invalidate_graph(h);
    }
    return DWG_OK;
}

int dwg_set_compensation(dwg_handle h, int on)
{
    if (!h) return DWG_ERR_INVALID;
    if (h->is_batch) return fail(h, DWG_ERR_STATE, "set the compensation per cloud handle");
    if (h->compensated != (on != 0)) {
        h->compensated = on != 0;
        invalidate_graph(h);
        ++h->bufgen;  // a captured graph holds the other kernels
    }
    return DWG_OK;
}

int dwg_set_update(dwg_handle h, int depth, int knn, int mode)
{
    if (!h) return DWG_ERR_INVALID;
    if (depth < 1 || depth > kMaxDepth) return fail(h, DWG_ERR_INVALID, "depth must be in [1, 14]");
    if (knn < 1 || knn > kMaxK) return fail(h, DWG_ERR_INVALID, "knn must be in [1, 32]");
    if (mode != DWG_UPDATE_LEVELSET && mode != DWG_UPDATE_DIRECT)
        return fail(h, DWG_ERR_INVALID, "mode must be DWG_UPDATE_LEVELSET or DWG_UPDATE_DIRECT");
    h->depth = depth;
    h->knn = knn;
    h->mode = mode;
    invalidate_graph(h);
    for (dwg_ctx *c : h->clouds) dwg_set_update(c, depth, knn, mode);
    return DWG_OK;
}

int dwg_set_tree(dwg_handle h, int path, float theta)
{
    if (!h) return DWG_ERR_INVALID;
    if (path != DWG_PATH_AUTO && path != DWG_PATH_ALLPAIRS && path != DWG_PATH_TREE)
        return fail(h, DWG_ERR_INVALID, "unknown path");
    if (!(theta > 0.f) || !(theta <= 1.f)) return fail(h, DWG_ERR_INVALID, "theta must be in (0, 1]");
    h->path = path;
    h->tree_beta = 1.0f / theta;
    invalidate_graph(h);
    for (dwg_ctx *c : h->clouds) dwg_set_tree(c, path, theta);
    return DWG_OK;
}

int dwg_set_weights(dwg_handle h, const float *a)
{
    if (!h || !a) return DWG_ERR_INVALID;
    cudaSetDevice(h->device);
    float *d = nullptr;
    DWG_CUDA_TRY(h, cudaMalloc(&d, h->n * sizeof(float)));
    int rc = upload(h, d, a, h->n * sizeof(float));
    if (!rc) {
        k_weights_in<<<nblk(h->n), 256, 0, h->stream>>>(d, h->d_perm, h->n, h->d_p4, h->d_err);
        rc = check_device_err(h);
        h->tree_built = false;  // node centres depend on the weights
        if (rc == DWG_ERR_NONFINITE) h->err = "weights must be finite and > 0";
    }
    cudaFree(d);
    return rc;
}

int dwg_set_regularization(dwg_handle h, int mode, int k, float vmin, float vmax,
                           float *delta_out)
{
    if (!h) return DWG_ERR_INVALID;
    cudaSetDevice(h->device);
    if (mode != DWG_REG_SOFTEN && mode != DWG_REG_CLAMP)
        return fail(h, DWG_ERR_INVALID, "mode must be DWG_REG_SOFTEN or DWG_REG_CLAMP");
    if (h->is_batch) return fail(h, DWG_ERR_STATE, "batch handles use the softened kernel");
    if (mode == DWG_REG_SOFTEN) {
        if (h->reg_mode != mode) {
            h->reg_mode = mode;
            ++h->delta_gen;
            invalidate_graph(h);
            ++h->bufgen;
        }
        return DWG_OK;
    }
    if (k < 1 || k > 31) return fail(h, DWG_ERR_INVALID, "k must be in [1, 31]");
    if (vmin == 0.f && vmax == 0.f) {
        // the paper's 0.0015 and 0.015 in a unit where the largest extent is 1
        const double ext = h->cube_L / 1.125;
        vmin = (float)(0.0015 * ext);
        vmax = (float)(0.015 * ext);
    }
    if (!(vmin > 0.f) || !(vmax >= vmin) || !isfinite(vmax))
        return fail(h, DWG_ERR_INVALID, "need 0 < vmin <= vmax (or both 0 for the defaults)");
    if (!h->d_delta2) DWG_CUDA_TRY(h, cudaMalloc(&h->d_delta2, h->n * sizeof(float)));
    if (!h->d_src16)
        DWG_CUDA_TRY(h, cudaMalloc(&h->d_src16, h->npad * kSrcFloatsClamp * sizeof(float)));
    float *d_out = nullptr;
    auto run = [&]() -> int {
        if (delta_out) DWG_CUDA_TRY(h, cudaMalloc(&d_out, h->n * sizeof(float)));
        if (launch_clamp_delta(h, k, (double)vmin, (double)vmax, d_out) != cudaSuccess)
            return fail(h, DWG_ERR_CUDA, "clamp radii launch failed");
        int r = check_device_err(h);
        if (r) return r;
        if (delta_out) return download(h, delta_out, d_out, h->n * sizeof(float));
        return DWG_OK;
    };
    int rc = run();
    if (!rc) {
        cudaError_t e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) rc = fail(h, DWG_ERR_CUDA, cudaGetErrorString(e));
    }
    cudaFree(d_out);
    if (rc) return rc;
    h->reg_mode = mode;
    ++h->delta_gen;  // tree opening radii and group lists depend on the radii
    // the records are repacked (with delta^2) before the next evaluation
    invalidate_graph(h);
    ++h->bufgen;  // a captured graph holds the other kernels and records
    return DWG_OK;
}

static int read_state(dwg_handle h, IterState *st);

int dwg_extract_level_set(dwg_handle h, float *tri_out, int64_t cap, int64_t *count,
                          double *iso_out)
{
    if (!h || !count || cap < 0) return DWG_ERR_INVALID;
    if (h->is_batch) return fail(h, DWG_ERR_STATE, "extract the level set per cloud handle");
    cudaSetDevice(h->device);
    int rc = engine_prepare(h);  // buffers, tree, records from the current normals
    if (rc) return rc;
    const bool tree = use_tree(h);
    if ((rc = ensure_levelset_buffers(h, tree))) return rc;
    unsigned long long *d_cnt = nullptr;
    float *d_tri = nullptr;
    auto body = [&]() -> int {
        DWG_CUDA_TRY(h, cudaMalloc(&d_cnt, sizeof(unsigned long long)));
        k_iter_reset<<<1, 1, 0, h->stream>>>(h->d_state, h->max_iters, nullptr);
        LAUNCH_CHECK(h);
        // w at the points -> w_bar; w at the corners
        if (tree) {
            if (launch_tree_moments(h) != cudaSuccess ||
                launch_tree_iter(h, h->lists_p, h->d_p4, h->n, true, h->d_part_p, h->n,
                                 h->d_state) != cudaSuccess ||
                launch_tree_iter(h, h->lists_c, h->d_corner_pos, h->ncorners, false, h->d_part_c,
                                 h->ncorners, h->d_state) != cudaSuccess)
                return fail(h, DWG_ERR_CUDA, "tree launch failed");
        } else {
            int r = eval_launch(h, h->d_p4, h->n, true, h->nchunks_p, h->d_part_p, h->n);
            if (!r) r = eval_launch(h, h->d_corner_pos, h->ncorners, false, h->nchunks_c,
                                    h->d_part_c, h->ncorners);
            if (r) return r;
        }
        if (launch_reduce_points(h, h->d_part_p, h->nchunks_p, h->n, h->d_p4, 1, true, h->d_wg,
                                 h->d_wsum_blocks) != cudaSuccess ||
            launch_iso(h) != cudaSuccess ||
            launch_reduce_w(h, h->d_part_c, h->nchunks_c, h->ncorners, h->d_wc) != cudaSuccess)
            return fail(h, DWG_ERR_CUDA, "reduce launch failed");
        DWG_CUDA_TRY(h, cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), h->stream));
        if (launch_mc_tris(h, nullptr, 0, d_cnt) != cudaSuccess)
            return fail(h, DWG_ERR_CUDA, "level-set launch failed");
        unsigned long long nt = 0;
        DWG_CUDA_TRY(h, cudaMemcpyAsync(&nt, d_cnt, sizeof nt, cudaMemcpyDeviceToHost, h->stream));
        DWG_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        *count = (int64_t)nt;
        if (iso_out) {
            IterState st;
            int r = read_state(h, &st);
            if (r) return r;
            *iso_out = st.iso;
        }
        if (!tri_out || (int64_t)nt > cap || nt == 0) return check_device_err(h);
        float *dst = tri_out;
        if (!is_device_ptr(tri_out)) {
            DWG_CUDA_TRY(h, cudaMalloc(&d_tri, nt * 9 * sizeof(float)));
            dst = d_tri;
        }
        DWG_CUDA_TRY(h, cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), h->stream));
        if (launch_mc_tris(h, dst, (int64_t)nt, d_cnt) != cudaSuccess)
            return fail(h, DWG_ERR_CUDA, "level-set launch failed");
        if (d_tri) {
            int r = download(h, tri_out, d_tri, nt * 9 * sizeof(float));
            if (r) return r;
        }
        DWG_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        return check_device_err(h);
    };
    rc = body();
    cudaStreamSynchronize(h->stream);
    cudaFree(d_cnt);
    cudaFree(d_tri);
    return rc;
}

int dwg_measure_fp32_peaks(int device, double *ffma_lane_ops_per_s, double *rsqrt_per_s,
                           double *ex2_per_s)
{
    if (!ffma_lane_ops_per_s || !rsqrt_per_s || !ex2_per_s) return DWG_ERR_INVALID;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return DWG_ERR_INVALID;
    return measure_fp32_peaks(device, ffma_lane_ops_per_s, rsqrt_per_s, ex2_per_s);
}

int dwg_selfcheck_wait(dwg_handle h, int polls)
{
    if (!h) return DWG_ERR_INVALID;
    if (polls < 1 || polls > (1 << 20)) return fail(h, DWG_ERR_INVALID, "polls must be in [1, 2^20]");
    cudaSetDevice(h->device);
    if (launch_wait_selfcheck(h, polls) != cudaSuccess)
        return fail(h, DWG_ERR_CUDA, "self-check launch failed");
    DWG_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return check_device_err(h);  // DWG_ERR_TIMEOUT, and the flag is cleared
}

int dwg_voronoi_weights(dwg_handle h, int m, float *a_out)
{
    if (!h) return DWG_ERR_INVALID;
    cudaSetDevice(h->device);
    if (m < 3 || m > 31) return fail(h, DWG_ERR_INVALID, "m must be in [3, 31]");
    if (h->is_batch) {
        for (size_t c = 0; c < h->clouds.size(); ++c) {
            int rc = dwg_voronoi_weights(h->clouds[c], m, a_out ? a_out + h->offsets[c] : nullptr);
            if (rc) return fail(h, rc, h->clouds[c]->err);
        }
        return DWG_OK;
    }
    int rc;
    double *scratch = nullptr;
    float *d_out = nullptr;
    auto run = [&]() -> int {
        DWG_CUDA_TRY(h, cudaMalloc(&scratch, (h->n + 1) * sizeof(double)));
        if (a_out) DWG_CUDA_TRY(h, cudaMalloc(&d_out, h->n * sizeof(float)));
        if (launch_voronoi_weights(h, m, scratch, d_out) != cudaSuccess)
            return fail(h, DWG_ERR_CUDA, "Voronoi weights launch failed");
        int r = check_device_err(h);
        if (r) return r;
        h->tree_built = false;  // node centres depend on the weights
        if (a_out) return download(h, a_out, d_out, h->n * sizeof(float));
        return DWG_OK;
    };
    rc = run();
    if (!rc) {
        cudaError_t e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) rc = fail(h, DWG_ERR_CUDA, cudaGetErrorString(e));
    }
    cudaFree(scratch);
    cudaFree(d_out);
    return rc;
}

static int normals_from_caller(dwg_handle h, const float *normals, float4 *dst)
{
    float *d = nullptr;
    DWG_CUDA_TRY(h, cudaMalloc(&d, h->n * 3 * sizeof(float)));
    int rc = upload(h, d, normals, h->n * 3 * sizeof(float));
    if (!rc) {
        k_normals_in<<<nblk(h->n), 256, 0, h->stream>>>(d, h->d_perm, h->n, dst, h->d_err);
        rc = check_device_err(h);
        if (rc == DWG_ERR_NONFINITE) h->err = "normals must be finite and non-zero";
    }
    cudaFree(d);
    return rc;
}

int dwg_set_init(dwg_handle h, int mode, uint64_t seed, const float *normals)
{
    if (!h) return DWG_ERR_INVALID;
    cudaSetDevice(h->device);
    if (h->is_batch) {
        if (mode == DWG_INIT_GIVEN)
            return fail(h, DWG_ERR_STATE, "batch handles take no DWG_INIT_GIVEN");
        // cloud c draws from seed + c
        for (size_t c = 0; c < h->clouds.size(); ++c) {
            int rc = dwg_set_init(h->clouds[c], mode, seed + c, normals);
            if (rc) return fail(h, rc, h->clouds[c]->err);
        }
        h->init_mode = mode;
        h->seed = seed;
        return DWG_OK;
    }
    if (mode == DWG_INIT_RANDOM || mode == DWG_INIT_PCA || mode == DWG_INIT_GAUSS) {
        h->init_mode = mode;
        h->seed = seed;
    } else if (mode == DWG_INIT_LEARNED) {
        if (!normals) return fail(h, DWG_ERR_INVALID, "DWG_INIT_LEARNED needs the parameters");
        if (!h->d_mlp_params)
            DWG_CUDA_TRY(h, cudaMalloc(&h->d_mlp_params, kMlpParamCount * sizeof(float)));
        int rc = upload(h, h->d_mlp_params, normals, kMlpParamCount * sizeof(float));
        if (rc) return rc;
        DWG_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        h->init_mode = mode;
        h->seed = seed;
    } else if (mode == DWG_INIT_GIVEN) {
        if (!normals) return fail(h, DWG_ERR_INVALID, "DWG_INIT_GIVEN needs normals");
        int rc = normals_from_caller(h, normals, h->d_nrm_init);
        if (rc) return rc;
        h->init_mode = mode;
    } else {
        return fail(h, DWG_ERR_INVALID, "unknown init mode");
    }
    h->normals_pending = true;
    return DWG_OK;
}

int dwg_set_normals(dwg_handle h, const float *normals)
{
    if (!h || !normals) return DWG_ERR_INVALID;
    cudaSetDevice(h->device);
    int rc = normals_from_caller(h, normals, h->d_nrm);
    if (rc) return rc;
    h->normals_pending = false;
    return DWG_OK;
}

int dwg_get_normals(dwg_handle h, float *normals_out)
{
    if (!h || !normals_out) return DWG_ERR_INVALID;
    cudaSetDevice(h->device);
    if (h->normals_pending) {
        int rc = prepare_normals(h);
        if (rc) return rc;
    }
    float *d = nullptr;
    DWG_CUDA_TRY(h, cudaMalloc(&d, h->n * 3 * sizeof(float)));
    k_normals_out<<<nblk(h->n), 256, 0, h->stream>>>(h->d_nrm, h->d_perm, h->n, d);
    int rc = download(h, normals_out, d, h->n * 3 * sizeof(float));
    cudaError_t e = cudaStreamSynchronize(h->stream);
    cudaFree(d);
    if (!rc && e != cudaSuccess) rc = fail(h, DWG_ERR_CUDA, cudaGetErrorString(e));
    return rc;
}

static int read_state(dwg_handle h, IterState *st)
{
    DWG_CUDA_TRY(h, cudaMemcpyAsync(st, h->d_state, sizeof(IterState), cudaMemcpyDeviceToHost,
                                    h->stream));
    DWG_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return DWG_OK;
}

int dwg_orient(dwg_handle h, float *normals_out, int *iters_out)
{
    if (!h) return DWG_ERR_INVALID;
    if (h->is_batch) return fail(h, DWG_ERR_STATE, "use dwg_orient_batch on a batch handle");
    cudaSetDevice(h->device);
    int rc = ensure_iter_buffers(h);
    if (rc) return rc;
    h->normals_pending = true;  // orient always starts from the initial normals
    if ((rc = prepare_normals(h))) return rc;
    k_iter_reset<<<1, 1, 0, h->stream>>>(h->d_state, h->max_iters, h->d_counter);
    LAUNCH_CHECK(h);
    if ((!h->graph_valid || h->graph_gen != h->bufgen) && (rc = build_graph(h))) return rc;
    cudaEvent_t e0, e1;
    DWG_CUDA_TRY(h, cudaEventCreate(&e0));
    DWG_CUDA_TRY(h, cudaEventCreate(&e1));
    cudaEventRecord(e0, h->stream);
    cudaError_t e = cudaGraphLaunch(h->graph_exec, h->stream);
    cudaEventRecord(e1, h->stream);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return fail(h, DWG_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
    }
    IterState st;
    rc = read_state(h, &st);
    h->stats.knn_deferred_last = st.ndefer;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if ((rc = check_device_err(h))) return rc;
    int it = std::min(st.iter, h->max_iters);
    h->tr_iso.assign(it, 0.0);
    h->tr_stat.assign(it, 0.0);
    h->tr_dn.assign(it, 0.0);
    h->tr_faces.assign(it, 0);
    if (it > 0) {
        std::vector<long long> tf(it);
        DWG_CUDA_TRY(h, cudaMemcpyAsync(h->tr_iso.data(), h->d_tr_iso, it * sizeof(double),
                                        cudaMemcpyDeviceToHost, h->stream));
        DWG_CUDA_TRY(h, cudaMemcpyAsync(h->tr_stat.data(), h->d_tr_stat, it * sizeof(double),
                                        cudaMemcpyDeviceToHost, h->stream));
        DWG_CUDA_TRY(h, cudaMemcpyAsync(h->tr_dn.data(), h->d_tr_dn, it * sizeof(double),
                                        cudaMemcpyDeviceToHost, h->stream));
        DWG_CUDA_TRY(h, cudaMemcpyAsync(tf.data(), h->d_tr_faces, it * sizeof(long long),
                                        cudaMemcpyDeviceToHost, h->stream));
        DWG_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        for (int i = 0; i < it; ++i) h->tr_faces[i] = tf[i];
    }
    h->stats.iters = it;
    h->stats.converged = st.done;
    h->stats.iso_last = st.iso;
    h->stats.stat_last = st.stat;
    h->stats.faces_last = it > 0 ? h->tr_faces[it - 1] : 0;
    h->stats.n_leaves = h->nleaves;
    h->stats.n_corners = h->ncorners;
    h->stats.interactions = interactions_per_iter(h) * it;
    if (use_tree(h)) {
        unsigned long long cnt = 0;
        DWG_CUDA_TRY(h, cudaMemcpy(&cnt, h->d_counter, sizeof(cnt), cudaMemcpyDeviceToHost));
        h->stats.interactions = (double)cnt;
    }
    h->stats.ms_orient = ms;
    if (iters_out) *iters_out = it;
    if (normals_out && (rc = dwg_get_normals(h, normals_out))) return rc;
    return st.done ? DWG_OK : DWG_NOT_CONVERGED;
}

int dwg_step(dwg_handle h, float *w_out, float *grad_out, float *dtheta_out, double *iso_out,
             double *stat_out)
{
    if (!h) return DWG_ERR_INVALID;
    if (h->is_batch) return fail(h, DWG_ERR_STATE, "use dwg_orient_batch on a batch handle");
    cudaSetDevice(h->device);
    int rc = ensure_iter_buffers(h);
    if (rc) return rc;
    if ((rc = prepare_normals(h))) return rc;
    k_iter_reset<<<1, 1, 0, h->stream>>>(h->d_state, h->max_iters, h->d_counter);
    LAUNCH_CHECK(h);
    cudaGraphConditionalHandle none = 0;
    if ((rc = enqueue_body(h, none, 0))) return rc;
    IterState st;
    if ((rc = read_state(h, &st))) return rc;
    if ((rc = check_device_err(h))) return rc;
    h->stats.knn_deferred_last = st.ndefer;
    if (iso_out) *iso_out = st.iso;
    if (stat_out) *stat_out = st.stat;
    if (!w_out && !grad_out && !dtheta_out) return DWG_OK;
    float *d = nullptr;
    DWG_CUDA_TRY(h, cudaMalloc(&d, h->n * 4 * sizeof(float)));
    if (w_out || grad_out) {
        k_wg_out<<<nblk(h->n), 256, 0, h->stream>>>(h->d_wg, h->d_perm, h->n, d, d + h->n);
        if (w_out && (rc = download(h, w_out, d, h->n * sizeof(float)))) goto out;
        if (grad_out && (rc = download(h, grad_out, d + h->n, 3 * h->n * sizeof(float)))) goto out;
    }
    if (dtheta_out) {
        DWG_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        k_scalar_out<<<nblk(h->n), 256, 0, h->stream>>>(h->d_dtheta, h->d_perm, h->n, d);
        if ((rc = download(h, dtheta_out, d, h->n * sizeof(float)))) goto out;
    }
out:
    cudaStreamSynchronize(h->stream);
    cudaFree(d);
    return rc;
}

int dwg_profile_step(dwg_handle h, float *ms_out, int cap, int *count)
{
    if (!h) return DWG_ERR_INVALID;
    cudaSetDevice(h->device);
    int rc = ensure_iter_buffers(h);
    if (rc) return rc;
    if ((rc = prepare_normals(h))) return rc;
    k_iter_reset<<<1, 1, 0, h->stream>>>(h->d_state, h->max_iters, h->d_counter);
    LAUNCH_CHECK(h);
    cudaEvent_t ev[10];
    for (int k = 0; k < 10; ++k) DWG_CUDA_TRY(h, cudaEventCreate(&ev[k]));
    unsigned long long *snap = nullptr, hs[2] = {0, 0};
    DWG_CUDA_TRY(h, cudaMalloc(&snap, 2 * sizeof(unsigned long long)));
    DWG_CUDA_TRY(h, cudaMemsetAsync(snap, 0, 2 * sizeof(unsigned long long), h->stream));
    cudaGraphConditionalHandle none = 0;
    rc = enqueue_body(h, none, 0, ev, snap);
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpy(hs, snap, sizeof(hs), cudaMemcpyDeviceToHost);
    cudaFree(snap);
    if (use_tree(h)) {
        h->stats.interactions_points_step = (double)hs[0];
        h->stats.interactions_corners_step =
            h->mode == DWG_UPDATE_LEVELSET ? (double)(hs[1] - hs[0]) : 0.0;
    } else {
        h->stats.interactions_points_step = (double)h->n * (double)h->n;
        h->stats.interactions_corners_step =
            h->mode == DWG_UPDATE_LEVELSET ? (double)h->ncorners * (double)h->n : 0.0;
    }
    float ms[9] = {0};
    for (int k = 0; k < 9; ++k) cudaEventElapsedTime(&ms[k], ev[k], ev[k + 1]);
    for (int k = 0; k < 10; ++k) cudaEventDestroy(ev[k]);
    if (rc) return rc;
    if (e != cudaSuccess) return fail(h, DWG_ERR_CUDA, cudaGetErrorString(e));
    if ((rc = check_device_err(h))) return rc;
    if (count) *count = 9;
    for (int k = 0; k < 9 && k < cap; ++k) ms_out[k] = ms[k];
    return DWG_OK;
}

int dwg_eval_gwn(dwg_handle h, const float *queries, int64_t m, float *w_out, float *grad_out)
{
    if (!h || !queries || !w_out) return DWG_ERR_INVALID;
    if (m < 1) return fail(h, DWG_ERR_INVALID, "m must be >= 1");
    cudaSetDevice(h->device);
    int rc;
    if ((rc = prepare_normals(h))) return rc;
    bool grad = grad_out != nullptr;
    float *qx = nullptr, *part = nullptr, *o = nullptr;
    float4 *q4 = nullptr, *wg = nullptr;
    auto body = [&]() -> int {
        DWG_CUDA_TRY(h, cudaMalloc(&qx, m * 3 * sizeof(float)));
        if ((rc = upload(h, qx, queries, m * 3 * sizeof(float)))) return rc;
        if (launch_check_finite(qx, 3 * m, h->d_err, h->stream) != cudaSuccess)
            return fail(h, DWG_ERR_CUDA, "finite-check launch failed");
        if ((rc = check_device_err(h))) return rc;
        DWG_CUDA_TRY(h, cudaMalloc(&q4, m * sizeof(float4)));
        k_xyz_to_f4<<<nblk(m), 256, 0, h->stream>>>(qx, m, q4);
        const bool tree = use_tree(h);
        int nch = tree ? 1 : eval_chunks(h, m, grad);
        DWG_CUDA_TRY(h, cudaMalloc(&part, (size_t)nch * (grad ? 8 : 2) * m * sizeof(float)));
        if (tree) {
            if ((rc = build_tree(h)) || (rc = tree_records(h))) return rc;
            DWG_CUDA_TRY(h, cudaMemsetAsync(h->d_counter, 0, sizeof(unsigned long long), h->stream));
            if (launch_tree_moments(h) != cudaSuccess ||
                launch_tree_gwn(h, q4, m, grad, part, m, nullptr) != cudaSuccess)
                return fail(h, DWG_ERR_CUDA, "tree launch failed");
        } else if ((rc = eval_launch(h, q4, m, grad, nch, part, m))) {
            return rc;
        }
        DWG_CUDA_TRY(h, cudaMalloc(&wg, m * sizeof(float4)));
        if (launch_reduce_points(h, part, nch, m, q4, grad ? 2 : 0, grad, wg, nullptr) !=
            cudaSuccess)
            return fail(h, DWG_ERR_CUDA, "reduce launch failed");
        DWG_CUDA_TRY(h, cudaMalloc(&o, m * 4 * sizeof(float)));
        k_wg_out<<<nblk(m), 256, 0, h->stream>>>(wg, nullptr, m, o, grad ? o + m : nullptr);
        if ((rc = download(h, w_out, o, m * sizeof(float)))) return rc;
        if (grad && (rc = download(h, grad_out, o + m, 3 * m * sizeof(float)))) return rc;
        DWG_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        h->stats.interactions_eval = (double)m * (double)h->n;
        if (tree) {
            unsigned long long cnt = 0;
            DWG_CUDA_TRY(h, cudaMemcpyAsync(&cnt, h->d_counter, sizeof(cnt), cudaMemcpyDeviceToHost,
                                            h->stream));
            DWG_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
            h->stats.interactions_eval = (double)cnt;
        }
        return check_device_err(h);
    };
    rc = body();
    cudaStreamSynchronize(h->stream);
    cudaFree(qx);
    cudaFree(q4);
    cudaFree(part);
    cudaFree(wg);
    cudaFree(o);
    return rc;
}

int dwg_autotune(dwg_handle h, int what, double w_budget, const char *cache_path,
                 dwg_tuning *out)
{
    if (!h) return DWG_ERR_INVALID;
    if (what & ~(DWG_TUNE_SHAPES | DWG_TUNE_TREE | DWG_TUNE_RELATIVE) ||
        !(what & (DWG_TUNE_SHAPES | DWG_TUNE_TREE)))
        return fail(h, DWG_ERR_INVALID,
                    "what: DWG_TUNE_SHAPES and/or DWG_TUNE_TREE, optionally DWG_TUNE_RELATIVE");
    if (h->reg_mode == DWG_REG_CLAMP)
        return fail(h, DWG_ERR_STATE, "the modified kernel has one evaluator shape and no tree: "
                                      "nothing to tune");
    cudaSetDevice(h->device);
    invalidate_graph(h);
    if (h->is_batch) {
        int64_t largest = -1;
        for (dwg_ctx *c : h->clouds) {
            c->stream = h->stream;
            dwg_tuning t;
            int rc = autotune(c, what, w_budget, cache_path, &t);
            if (rc) return fail(h, rc, "cloud: " + c->err);
            if (c->n > largest) {
                largest = c->n;
                if (out) *out = t;
            }
        }
        return DWG_OK;
    }
    return autotune(h, what, w_budget, cache_path, out);
}

int dwg_get_tuning(dwg_handle h, dwg_tuning *out)
{
    if (!h || !out) return DWG_ERR_INVALID;
    if (h->is_batch) {  // the largest cloud's settings
        const dwg_ctx *big = h->clouds.empty() ? h : h->clouds[0];
        for (const dwg_ctx *c : h->clouds)
            if (c->n > big->n) big = c;
        tuning_of(big, out);
        return DWG_OK;
    }
    tuning_of(h, out);
    return DWG_OK;
}

int dwg_set_tuning(dwg_handle h, const dwg_tuning *t)
{
    if (!h || !t) return DWG_ERR_INVALID;
    invalidate_graph(h);
    if (h->is_batch) {
        for (dwg_ctx *c : h->clouds) {
            int rc = apply_tuning(c, t);
            if (rc) return fail(h, rc, c->err);
        }
        return DWG_OK;
    }
    return apply_tuning(h, t);
}

int dwg_get_stats(dwg_handle h, dwg_stats *out)
{
    if (!h || !out) return DWG_ERR_INVALID;
    *out = h->stats;
    out->n_points = h->n;
    return DWG_OK;
}

int dwg_get_trace(dwg_handle h, double *iso, double *stat, double *mean_dn, int64_t *faces,
                  int cap, int *count)
{
    if (!h) return DWG_ERR_INVALID;
    int it = (int)h->tr_iso.size();
    if (count) *count = it;
    for (int i = 0; i < it && i < cap; ++i) {
        if (iso) iso[i] = h->tr_iso[i];
        if (stat) stat[i] = h->tr_stat[i];
        if (mean_dn) mean_dn[i] = h->tr_dn[i];
        if (faces) faces[i] = h->tr_faces[i];
    }
    return DWG_OK;
}

int dwg_get_leaves(dwg_handle h, int64_t *leaves_out, int64_t cap, int64_t *count)
{
    if (!h || !count) return DWG_ERR_INVALID;
    cudaSetDevice(h->device);
    int rc = build_discretization(h, h->depth);
    if (rc) return rc;
    *count = h->nleaves;
    if (!leaves_out || cap < h->nleaves) return DWG_OK;
    std::vector<int4> L(h->nleaves);
    DWG_CUDA_TRY(h, cudaMemcpyAsync(L.data(), h->d_leaves, h->nleaves * sizeof(int4),
                                    cudaMemcpyDeviceToHost, h->stream));
    DWG_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    std::vector<int64_t> rec(5 * h->nleaves);
    for (int64_t i = 0; i < h->nleaves; ++i) {
        uint64_t code = (uint64_t)(uint32_t)L[i].y | ((uint64_t)(uint32_t)L[i].z << 32);
        rec[5 * i] = L[i].x;
        rec[5 * i + 1] = (int64_t)compact3(code);
        rec[5 * i + 2] = (int64_t)compact3(code >> 1);
        rec[5 * i + 3] = (int64_t)compact3(code >> 2);
        rec[5 * i + 4] = L[i].w;
    }
    std::vector<int64_t> order(h->nleaves);
    for (int64_t i = 0; i < h->nleaves; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
        for (int k = 0; k < 4; ++k)
            if (rec[5 * a + k] != rec[5 * b + k]) return rec[5 * a + k] < rec[5 * b + k];
        return false;
    });
    std::vector<int64_t> sorted(5 * h->nleaves);
    for (int64_t i = 0; i < h->nleaves; ++i)
        for (int k = 0; k < 5; ++k) sorted[5 * i + k] = rec[5 * order[i] + k];
    return download(h, leaves_out, sorted.data(), sorted.size() * sizeof(int64_t)) ||
                   cudaStreamSynchronize(h->stream)
               ? DWG_ERR_CUDA
               : DWG_OK;
}

int dwg_get_corners(dwg_handle h, int64_t *keys_out, int64_t cap, int64_t *count)
{
    if (!h || !count) return DWG_ERR_INVALID;
    cudaSetDevice(h->device);
    int rc = build_discretization(h, h->depth);
    if (rc) return rc;
    *count = h->ncorners;
    if (!keys_out || cap < h->ncorners) return DWG_OK;
    std::vector<uint64_t> K(h->ncorners);
    DWG_CUDA_TRY(h, cudaMemcpyAsync(K.data(), h->d_corner_keys, h->ncorners * sizeof(uint64_t),
                                    cudaMemcpyDeviceToHost, h->stream));
    DWG_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    const int64_t S1 = ((int64_t)1 << h->depth) + 1;
    std::vector<int64_t> out(h->ncorners);
    for (int64_t i = 0; i < h->ncorners; ++i) {
        int64_t X = (int64_t)compact3(K[i]), Y = (int64_t)compact3(K[i] >> 1),
                Z = (int64_t)compact3(K[i] >> 2);
        out[i] = (X * S1 + Y) * S1 + Z;
    }
    std::sort(out.begin(), out.end());
    return download(h, keys_out, out.data(), out.size() * sizeof(int64_t)) ||
                   cudaStreamSynchronize(h->stream)
               ? DWG_ERR_CUDA
               : DWG_OK;
}

int dwg_get_tree(dwg_handle h, int64_t cap, int64_t *nodes_out, int *leaf_out, int64_t *perm_out,
                 double *area_out, double *centre_out, double *radius_out, float *record_out)
{
    if (!h || !nodes_out || !leaf_out) return DWG_ERR_INVALID;
    if (h->is_batch) return fail(h, DWG_ERR_STATE, "read the tree of a cloud handle");
    cudaSetDevice(h->device);
    int rc;
    if ((rc = build_tree(h)) || (rc = tree_records(h))) return rc;
    const int64_t nn = (int64_t)2 << h->tree_levels;
    *nodes_out = nn;
    *leaf_out = h->tree_leaf;
    if (cap < nn) return DWG_OK;
    if (perm_out && (rc = download(h, perm_out, h->d_perm, h->n * sizeof(int64_t)))) return rc;
    if (area_out && (rc = download(h, area_out, h->d_tree_A, nn * sizeof(double)))) return rc;
    if (centre_out && (rc = download(h, centre_out, h->d_tree_C, 3 * nn * sizeof(double))))
        return rc;
    if (radius_out && (rc = download(h, radius_out, h->d_tree_R, nn * sizeof(double)))) return rc;
    if (record_out && (rc = download(h, record_out, h->d_tree_rec, nn * sizeof(float4))))
        return rc;
    DWG_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return check_device_err(h);
}

int dwg_mlp_features(dwg_handle h, float *X_out)
{
    if (!h || !X_out) return DWG_ERR_INVALID;
    if (h->is_batch) return fail(h, DWG_ERR_STATE, "not on a batch handle");
    cudaSetDevice(h->device);
    float *X = nullptr;
    double *cR = nullptr;
    auto run = [&]() -> int {
        DWG_CUDA_TRY(h, cudaMalloc(&X, h->n * 64 * sizeof(float)));
        DWG_CUDA_TRY(h, cudaMalloc(&cR, 4 * sizeof(double)));
        if (launch_features(h, X, true, cR) != cudaSuccess)
            return fail(h, DWG_ERR_CUDA, "features launch failed");
        int rc = download(h, X_out, X, h->n * 64 * sizeof(float));
        if (rc) return rc;
        DWG_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        return check_device_err(h);
    };
    int rc = run();
    cudaFree(X);
    cudaFree(cR);
    return rc;
}

static int mlp_check(std::initializer_list<const void *> ptrs, int64_t B)
{
    for (const void *p : ptrs)
        if (!p || !is_device_ptr(p)) {
            set_global_error("dwg_mlp_*: every array must be device memory");
            return DWG_ERR_INVALID;
        }
    if (B < 1) {
        set_global_error("dwg_mlp_*: B must be >= 1");
        return DWG_ERR_INVALID;
    }
    return DWG_OK;
}

static int mlp_finish(cudaError_t e, cudaStream_t s)
{
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_global_error(std::string("dwg_mlp_*: ") + cudaGetErrorString(e));
        return DWG_ERR_CUDA;
    }
    return DWG_OK;
}

int dwg_mlp_forward(const float *params, const float *X, int64_t B, float *Y, void *stream)
{
    int rc = mlp_check({params, X, Y}, B);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    rc = mlp_finish(launch_mlp_forward(params, X, B, Y, s, nullptr), s);
    if (rc) return rc;
    if (mlp_forward_error(s) != 0) {
        set_global_error("dwg_mlp_forward: a tensor-core wait gave up");
        return DWG_ERR_TIMEOUT;
    }
    return DWG_OK;
}

int dwg_mlp_grad(const float *params, const float *X, const float *T, int64_t B, float *grad,
                 double *loss, void *stream)
{
    int rc = mlp_check({params, X, T, grad}, B);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    double *dl = nullptr;
    cudaError_t e = cudaMallocAsync(&dl, sizeof(double), s);
    if (e == cudaSuccess) e = launch_mlp_grad(params, X, T, B, grad, dl, s);
    double hl = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hl, dl, sizeof(double), cudaMemcpyDeviceToHost, s);
    rc = mlp_finish(e, s);
    cudaFreeAsync(dl, s);
    cudaStreamSynchronize(s);
    if (loss) *loss = hl;
    return rc;
}

int dwg_mlp_adam(float *params, const float *grad, float *m, float *v, int step, float lr,
                 void *stream)
{
    int rc = mlp_check({params, grad, m, v}, 1);
    if (rc) return rc;
    if (step < 1 || !(lr > 0.f)) {
        set_global_error("dwg_mlp_adam: need step >= 1 and lr > 0");
        return DWG_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    return mlp_finish(launch_adam(params, grad, m, v, step, lr, s), s);
}

int dwg_knn(dwg_handle h, const float *queries, int64_t m, int k, int64_t *idx_out)
{
    if (!h || !queries || !idx_out) return DWG_ERR_INVALID;
    if (m < 1 || k < 1 || k > kMaxK) return fail(h, DWG_ERR_INVALID, "need m >= 1, 1 <= k <= 32");
    cudaSetDevice(h->device);
    float *qx = nullptr;
    float4 *q4 = nullptr;
    int64_t *idx = nullptr;
    int rc;
    auto body = [&]() -> int {
        DWG_CUDA_TRY(h, cudaMalloc(&qx, m * 3 * sizeof(float)));
        if ((rc = upload(h, qx, queries, m * 3 * sizeof(float)))) return rc;
        DWG_CUDA_TRY(h, cudaMalloc(&q4, m * sizeof(float4)));
        k_xyz_to_f4<<<nblk(m), 256, 0, h->stream>>>(qx, m, q4);
        DWG_CUDA_TRY(h, cudaMalloc(&idx, m * k * sizeof(int64_t)));
        if (launch_knn_query(h, q4, m, k, idx) != cudaSuccess)
            return fail(h, DWG_ERR_CUDA, "knn launch failed");
        if ((rc = download(h, idx_out, idx, m * k * sizeof(int64_t)))) return rc;
        DWG_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        return check_device_err(h);
    };
    rc = body();
    cudaStreamSynchronize(h->stream);
    cudaFree(qx);
    cudaFree(q4);
    cudaFree(idx);
    return rc;
}

// ---------------------------------------------------------------------------
// batches: many clouds, one launch per iteration for the all-pairs sums
// ---------------------------------------------------------------------------
__global__ void k_batch_cond(IterState *const *states, int nc, int max_iters,
                             cudaGraphConditionalHandle cond)
{
    __shared__ int s_more;
    if (threadIdx.x == 0) s_more = 0;
    __syncthreads();
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
        const IterState *st = states[c];
        if (!st->done && st->iter < max_iters) s_more = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) cudaGraphSetConditional(cond, s_more ? 1u : 0u);
}

// per-cloud octree depth when none is set: about half the bits of n
static int auto_depth(int64_t n)
{
    int d = (int)lround(0.5 * log2((double)std::max<int64_t>(n, 2)));
    return std::min(10, std::max(5, d));
}

static int batch_prepare(dwg_ctx *h)
{
    for (dwg_ctx *c : h->clouds) {
        c->stream = h->stream;
        int rc = ensure_iter_buffers(c);
        if (rc) return fail(h, rc, "cloud: " + c->err);
        c->normals_pending = true;
        if ((rc = prepare_normals(c))) return fail(h, rc, "cloud: " + c->err);
        k_iter_reset<<<1, 1, 0, h->stream>>>(c->d_state, c->max_iters, c->d_counter);
    }
    LAUNCH_CHECK(h);
    return DWG_OK;
}

// Blocks of a cloud's part of a batched phase: the grid its own launch uses
// (launch_reduce_points, launch_reduce_w, launch_mc_faces,
// launch_knn_scatter, launch_normal_update, launch_select, the tree phases).
static int phase_blocks(const dwg_ctx *c, int ph)
{
    const bool ls = c->mode == DWG_UPDATE_LEVELSET;
    switch (ph) {
    case kPhReducePoints: return (int)ceil_div(c->n, 256);
    case kPhReduceW: return ls ? (int)ceil_div(c->ncorners, 256) : 0;
    case kPhMcFaces: return ls ? (int)ceil_div(c->nleaves, 256) : 0;
    case kPhKnn: return ls ? (int)ceil_div(c->max_faces, 128) : 0;
    case kPhKnnDefer: return ls ? 8 : 0;  // blocks take the cloud's deferred faces in turn
    case kPhUpdate: return (int)ceil_div(c->n, 256);
    case kPhSelHist:
    case kPhSelSum: return select_blocks(c->n);
    case kPhIso:
    case kPhSelFind:
    case kPhSelFinal: return 1;
    default: return tree_phase_blocks(c, ph, -1);
    }
}

// The batched iteration's tables: each cloud's arguments and the block
// offsets of every phase.  The batched phases need one kernel instance for
// all clouds: the same k (10) and the softened kernel everywhere; otherwise
// the clouds' chains run as separate graph branches.
static int batch_plan(dwg_ctx *h)
{
    const int ncl = (int)h->clouds.size();
    h->batched = false;
    h->lanes.clear();
    if (!h->batch_phases) return DWG_OK;
    for (const dwg_ctx *c : h->clouds)
        if (c->knn != 10 || c->reg_mode != DWG_REG_SOFTEN) return DWG_OK;
    // lanes balanced by an estimate of each cloud's per-iteration work
    // (largest first onto the least loaded lane); a tree cloud's list
    // evaluations dominate its share, an all-pairs cloud's sums run in the
    // shared launch before the lanes
    const int nl = std::min(h->batch_phases, ncl);
    h->lanes.assign(nl, dwg_ctx::Lane());
    std::vector<int> order(ncl);
    for (int i = 0; i < ncl; ++i) order[i] = i;
    auto work = [&](int i) {
        const dwg_ctx *c = h->clouds[i];
        return (double)c->n * (use_tree(c) ? 32.0 : 1.0);
    };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work(a) > work(b); });
    std::vector<double> load(nl, 0.0);
    for (int i : order) {
        const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        load[l] += work(i);
        h->lanes[l].clouds.push_back(h->clouds[i]);
    }
    std::vector<CloudIter> tab;
    std::vector<int> off;
    for (auto &L : h->lanes) {
        const int m = (int)L.clouds.size();
        L.base = (int)tab.size();
        L.off_base = off.size();
        int maxL = 0;
        for (dwg_ctx *c : L.clouds) {
            tab.emplace_back();
            fill_cloud_iter(c, &tab.back());
            if (use_tree(c)) {
                maxL = std::max(maxL, c->tree_levels);
                if (!tree_lists_current(c, false)) L.walk_p.push_back(c);
                if (c->mode == DWG_UPDATE_LEVELSET && !tree_lists_current(c, true))
                    L.walk_c.push_back(c);
            }
        }
        const int rows = kPhCount + maxL;
        L.lv_blocks.assign(maxL, 0);
        for (int r = 0; r < rows; ++r) {
            const size_t row0 = off.size();
            off.push_back(0);
            for (int i = 0; i < m; ++i) {
                const dwg_ctx *c = L.clouds[i];
                const int b =
                    r < kPhCount ? phase_blocks(c, r) : tree_phase_blocks(c, 0, r - kPhCount);
                off.push_back(off[row0 + i] + b);
            }
            if (r < kPhCount) L.ph_blocks[r] = off.back();
            else L.lv_blocks[r - kPhCount] = off.back();
        }
    }
    cudaFree(h->d_citer);
    cudaFree(h->d_boff);
    h->d_citer = nullptr;
    h->d_boff = nullptr;
    DWG_CUDA_TRY(h, cudaMalloc(&h->d_citer, tab.size() * sizeof(CloudIter)));
    DWG_CUDA_TRY(h, cudaMemcpy(h->d_citer, tab.data(), tab.size() * sizeof(CloudIter),
                               cudaMemcpyHostToDevice));
    DWG_CUDA_TRY(h, cudaMalloc(&h->d_boff, off.size() * sizeof(int)));
    DWG_CUDA_TRY(h, cudaMemcpy(h->d_boff, off.data(), off.size() * sizeof(int),
                               cudaMemcpyHostToDevice));
    h->batched = true;
    return DWG_OK;
}

static int batch_tables(dwg_ctx *h)
{
    std::vector<GwnCloud> cp, cc;
    std::vector<GwnItem> ip, ic;
    for (dwg_ctx *c : h->clouds) {
        if (use_tree(c)) continue;
        EvalParams ep = make_eval_params(c);
        int64_t ntiles = c->npad / kSrcTile;
        for (int pass = 0; pass < 2; ++pass) {
            bool grad = pass == 0;
            if (!grad && c->mode != DWG_UPDATE_LEVELSET) continue;
            int64_t m = grad ? c->n : c->ncorners;
            int nch = grad ? c->nchunks_p : c->nchunks_c;
            GwnCloud g;
            g.src = c->d_src;
            g.ntiles = ntiles;
            g.q = grad ? c->d_p4 : c->d_corner_pos;
            g.m = m;
            g.tpc = (int)ceil_div(ntiles, nch);
            g.part = grad ? c->d_part_p : c->d_part_c;
            g.stride = m;
            g.ep = ep;
            g.st = c->d_state;
            auto &tab = grad ? cp : cc;
            auto &its = grad ? ip : ic;
            int id = (int)tab.size();
            tab.push_back(g);
            int64_t qt = ceil_div(m, batch_query_tile(grad));
            for (int ch = 0; ch < nch; ++ch)
                for (int64_t t = 0; t < qt; ++t) its.push_back(GwnItem{id, (int)t, ch, 0});
        }
    }
    auto put = [&](auto &vec, auto **dptr) -> int {
        cudaFree(*dptr);
        *dptr = nullptr;
        if (vec.empty()) return DWG_OK;
        DWG_CUDA_TRY(h, cudaMalloc(dptr, vec.size() * sizeof(vec[0])));
        DWG_CUDA_TRY(h, cudaMemcpy(*dptr, vec.data(), vec.size() * sizeof(vec[0]),
                                   cudaMemcpyHostToDevice));
        return DWG_OK;
    };
    int rc;
    if ((rc = put(cp, &h->d_bcl_p)) || (rc = put(cc, &h->d_bcl_c)) || (rc = put(ip, &h->d_bit_p)) ||
        (rc = put(ic, &h->d_bit_c)))
        return rc;
    h->nit_p = (int64_t)ip.size();
    h->nit_c = (int64_t)ic.size();
    std::vector<IterState *> st;
    for (dwg_ctx *c : h->clouds) st.push_back(c->d_state);
    cudaFree(h->d_states);
    h->d_states = nullptr;
    DWG_CUDA_TRY(h, cudaMalloc(&h->d_states, st.size() * sizeof(IterState *)));
    DWG_CUDA_TRY(h, cudaMemcpy(h->d_states, st.data(), st.size() * sizeof(IterState *),
                               cudaMemcpyHostToDevice));
    return batch_plan(h);
}

// one iteration of every cloud, phase by phase: each phase is one launch
// over every cloud's blocks (the all-pairs sums, the Barnes-Hut moments per
// tree level, the list evaluations and their combination, the reduce, the
// iso-value, the level set, the kNN scatter, the update and the convergence
// select), so the number of launches per iteration does not grow with the
// number of clouds.  Each cloud's blocks are those of its own launch: the
// results are the same bits as orienting the cloud alone.  Tree clouds whose
// interaction lists are not resident (they would not fit) walk the tree in
// launches of their own.
static cudaError_t batch_lane_phases(dwg_ctx *h, const dwg_ctx::Lane &L, bool scr,
                                     cudaStream_t s)
{
    const int ncl = (int)L.clouds.size();
    const CloudIter *cl = h->d_citer + L.base;
    const int *ph = L.ph_blocks;
    auto off = [&](int row) { return h->d_boff + L.off_base + (size_t)row * (ncl + 1); };
    cudaError_t e = cudaSuccess;
    auto ok = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
    // Barnes-Hut moments: leaves, then each tree level from the bottom up
    ok(launch_tree_batch(kPhLeafMom, cl, off(kPhLeafMom), ncl, ph[kPhLeafMom], -1, scr, s));
    for (int lv = (int)L.lv_blocks.size() - 1; lv >= 0; --lv)
        ok(launch_tree_batch(kPhLeafMom, cl, off(kPhCount + lv), ncl, L.lv_blocks[lv], lv, scr, s));
    ok(launch_tree_batch(kPhMomRec, cl, off(kPhMomRec), ncl, ph[kPhMomRec], -1, scr, s));
    // w and grad w at the points
    ok(launch_tree_batch(kPhListsP, cl, off(kPhListsP), ncl, ph[kPhListsP], -1, scr, s));
    ok(launch_tree_batch(kPhCombineP, cl, off(kPhCombineP), ncl, ph[kPhCombineP], -1, scr, s));
    for (dwg_ctx *c : L.walk_p) {
        c->stream = s;
        ok(launch_tree_iter(c, c->lists_p, c->d_p4, c->n, true, c->d_part_p, c->n, c->d_state));
    }
    ok(launch_eval_batch(kPhReducePoints, cl, off(kPhReducePoints), ncl, ph[kPhReducePoints], s));
    ok(launch_iter_batch(kPhIso, cl, off(kPhIso), ncl, ph[kPhIso], 0, s));
    // w at the corners, level set, face gradients to the k nearest points
    ok(launch_tree_batch(kPhListsC, cl, off(kPhListsC), ncl, ph[kPhListsC], -1, scr, s));
    ok(launch_tree_batch(kPhCombineC, cl, off(kPhCombineC), ncl, ph[kPhCombineC], -1, scr, s));
    for (dwg_ctx *c : L.walk_c) {
        c->stream = s;
        ok(launch_tree_iter(c, c->lists_c, c->d_corner_pos, c->ncorners, false, c->d_part_c,
                            c->ncorners, c->d_state));
    }
    ok(launch_eval_batch(kPhReduceW, cl, off(kPhReduceW), ncl, ph[kPhReduceW], s));
    ok(launch_iter_batch(kPhMcFaces, cl, off(kPhMcFaces), ncl, ph[kPhMcFaces], 0, s));
    ok(launch_iter_batch(kPhKnn, cl, off(kPhKnn), ncl, ph[kPhKnn], 0, s));
    ok(launch_iter_batch(kPhKnnDefer, cl, off(kPhKnnDefer), ncl, ph[kPhKnnDefer], 0, s));
    // normal update and convergence
    ok(launch_iter_batch(kPhUpdate, cl, off(kPhUpdate), ncl, ph[kPhUpdate], 0, s));
    for (int level = 0; level < 3; ++level) {
        ok(launch_iter_batch(kPhSelHist, cl, off(kPhSelHist), ncl, ph[kPhSelHist], level, s));
        ok(launch_iter_batch(kPhSelFind, cl, off(kPhSelFind), ncl, ph[kPhSelFind], level, s));
    }
    ok(launch_iter_batch(kPhSelSum, cl, off(kPhSelSum), ncl, ph[kPhSelSum], 0, s));
    ok(launch_iter_batch(kPhSelFinal, cl, off(kPhSelFinal), ncl, ph[kPhSelFinal], 0, s));
    return e;
}

static int batch_body_phases(dwg_ctx *h)
{
    const bool scr = h->kernel == DWG_KERNEL_SCREENED && h->lambda > 0.f;
    cudaStream_t s = h->stream;
    if (launch_gwn_batch(h->d_bcl_p, h->d_bit_p, h->nit_p, true, scr, h->d_err, s) !=
            cudaSuccess ||
        launch_gwn_batch(h->d_bcl_c, h->d_bit_c, h->nit_c, false, scr, h->d_err, s) !=
            cudaSuccess)
        return fail(h, DWG_ERR_CUDA, "batched gwn launch failed");
    if (h->lanes.size() == 1) {
        cudaError_t e = batch_lane_phases(h, h->lanes[0], scr, s);
        if (e != cudaSuccess)
            return fail(h, DWG_ERR_CUDA, std::string("batched phase launch: ") + cudaGetErrorString(e));
        return DWG_OK;
    }
    // each lane on the stream of its first cloud, forked from and joined
    // back into the batch stream
    if (!h->ev_fork)
        DWG_CUDA_TRY(h, cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    DWG_CUDA_TRY(h, cudaEventRecord(h->ev_fork, s));
    for (const auto &L : h->lanes) {
        dwg_ctx *c0 = L.clouds[0];
        if (!c0->ev_join)
            DWG_CUDA_TRY(h, cudaEventCreateWithFlags(&c0->ev_join, cudaEventDisableTiming));
        DWG_CUDA_TRY(h, cudaStreamWaitEvent(c0->own_stream, h->ev_fork, 0));
        cudaError_t e = batch_lane_phases(h, L, scr, c0->own_stream);
        if (e != cudaSuccess)
            return fail(h, DWG_ERR_CUDA, std::string("batched phase launch: ") + cudaGetErrorString(e));
        DWG_CUDA_TRY(h, cudaEventRecord(c0->ev_join, c0->own_stream));
        DWG_CUDA_TRY(h, cudaStreamWaitEvent(s, c0->ev_join, 0));
    }
    return DWG_OK;
}

// one iteration of every cloud when the phases cannot be batched (mixed k
// or kernels): the all-pairs sums of every cloud in one launch, then each
// cloud's chain (tree sums, reduce, iso-value, level set,
// kNN scatter, update, convergence) on the cloud's own stream, forked from
// and joined back into the batch stream, so that the chains of different
// clouds run concurrently (one graph branch per cloud)
static int batch_body_branches(dwg_ctx *h, cudaGraphConditionalHandle cond)
{
    bool scr = h->kernel == DWG_KERNEL_SCREENED && h->lambda > 0.f;
    if (launch_gwn_batch(h->d_bcl_p, h->d_bit_p, h->nit_p, true, scr, h->d_err, h->stream) !=
            cudaSuccess ||
        launch_gwn_batch(h->d_bcl_c, h->d_bit_c, h->nit_c, false, scr, h->d_err, h->stream) !=
            cudaSuccess)
        return fail(h, DWG_ERR_CUDA, "batched gwn launch failed");
    if (!h->ev_fork)
        DWG_CUDA_TRY(h, cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    DWG_CUDA_TRY(h, cudaEventRecord(h->ev_fork, h->stream));
    for (dwg_ctx *c : h->clouds) {
        if (!c->ev_join)
            DWG_CUDA_TRY(h, cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
        DWG_CUDA_TRY(h, cudaStreamWaitEvent(c->own_stream, h->ev_fork, 0));
        c->stream = c->own_stream;
        if (use_tree(c)) {
            if (launch_tree_moments(c) != cudaSuccess ||
                launch_tree_iter(c, c->lists_p, c->d_p4, c->n, true, c->d_part_p, c->n,
                                 c->d_state) != cudaSuccess ||
                (c->mode == DWG_UPDATE_LEVELSET &&
                 launch_tree_iter(c, c->lists_c, c->d_corner_pos, c->ncorners, false, c->d_part_c,
                                  c->ncorners, c->d_state) != cudaSuccess))
                return fail(h, DWG_ERR_CUDA, "tree launch failed");
        }
        if (launch_reduce_points(c, c->d_part_p, c->nchunks_p, c->n, c->d_p4, 1, true, c->d_wg,
                                 c->d_wsum_blocks) != cudaSuccess ||
            launch_iso(c) != cudaSuccess)
            return fail(h, DWG_ERR_CUDA, "reduce launch failed");
        if (c->mode == DWG_UPDATE_LEVELSET &&
            (launch_reduce_w(c, c->d_part_c, c->nchunks_c, c->ncorners, c->d_wc) != cudaSuccess ||
             launch_mc_faces(c) != cudaSuccess || launch_knn_scatter(c) != cudaSuccess))
            return fail(h, DWG_ERR_CUDA, "level-set launch failed");
        if (launch_normal_update(c) != cudaSuccess || launch_select(c, cond, 0) != cudaSuccess)
            return fail(h, DWG_ERR_CUDA, "update launch failed");
        DWG_CUDA_TRY(h, cudaEventRecord(c->ev_join, c->stream));
        DWG_CUDA_TRY(h, cudaStreamWaitEvent(h->stream, c->ev_join, 0));
    }
    return DWG_OK;
}

static int batch_body(dwg_ctx *h, cudaGraphConditionalHandle cond)
{
    int rc = h->batched ? batch_body_phases(h) : batch_body_branches(h, cond);
    if (rc) return rc;
    k_batch_cond<<<1, 256, 0, h->stream>>>(h->d_states, (int)h->clouds.size(), h->max_iters, cond);
    LAUNCH_CHECK(h);
    return DWG_OK;
}

// buffers of every cloud that the batch graph refers to
static uint64_t batch_gen(const dwg_ctx *h)
{
    uint64_t g = h->bufgen;
    for (const dwg_ctx *c : h->clouds) g = g * 1000003ull + c->bufgen;
    return g;
}

static int batch_build_graph(dwg_ctx *h)
{
    invalidate_graph(h);
    int rc = batch_tables(h);
    if (rc) return rc;
    cudaGraph_t g = nullptr;
    DWG_CUDA_TRY(h, cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle cond;
    cudaError_t e = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return fail(h, DWG_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(e));
    }
    cudaStream_t saved = h->stream;
    h->stream = h->own_stream;
    e = cudaStreamBeginCaptureToGraph(h->stream, cp.conditional.phGraph_out[0], nullptr, nullptr,
                                      0, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
        h->stream = saved;
        cudaGraphDestroy(g);
        return fail(h, DWG_ERR_CUDA, std::string("begin capture: ") + cudaGetErrorString(e));
    }
    rc = batch_body(h, cond);
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(h->stream, &captured);
    if (!rc && e == cudaSuccess)
        h->stats.kernels_per_iteration = count_kernel_nodes(cp.conditional.phGraph_out[0]);
    h->stream = saved;
    for (dwg_ctx *c : h->clouds) c->stream = saved;
    if (rc || e != cudaSuccess) {
        cudaGraphDestroy(g);
        if (rc) return rc;
        return fail(h, DWG_ERR_CUDA, std::string("end capture: ") + cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&h->graph_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        h->graph_exec = nullptr;
        return fail(h, DWG_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e));
    }
    h->graph_valid = true;
    h->graph_gen = batch_gen(h);
    return DWG_OK;
}

int dwg_create_batch(const float *points, const int64_t *offsets, int n_clouds, dwg_handle *out)
{
    if (out) *out = nullptr;
    if (!out || !points || !offsets || n_clouds < 1) {
        set_global_error("dwg_create_batch: null argument or n_clouds < 1");
        return DWG_ERR_INVALID;
    }
    std::vector<int64_t> off(n_clouds + 1);
    if (!is_host_ptr(offsets)) {
        if (cudaMemcpy(off.data(), offsets, off.size() * sizeof(int64_t), cudaMemcpyDefault) !=
            cudaSuccess) {
            set_global_error("dwg_create_batch: cannot read offsets");
            return DWG_ERR_CUDA;
        }
    } else {
        memcpy(off.data(), offsets, off.size() * sizeof(int64_t));
    }
    if (off[0] != 0) {
        set_global_error("dwg_create_batch: offsets[0] must be 0");
        return DWG_ERR_INVALID;
    }
    for (int c = 0; c < n_clouds; ++c)
        if (off[c + 1] <= off[c]) {
            set_global_error("dwg_create_batch: every cloud needs at least one point");
            return DWG_ERR_INVALID;
        }
    const int64_t total = off[n_clouds];
    dwg_ctx *h = new (std::nothrow) dwg_ctx();
    if (!h) return DWG_ERR_OOM;
    h->is_batch = true;
    h->offsets = off;
    float *dpts = nullptr;
    bool own = false;
    auto body = [&]() -> int {
        DWG_CUDA_TRY(h, cudaGetDevice(&h->device));
        DWG_CUDA_TRY(h, cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking));
        h->stream = h->own_stream;
        DWG_CUDA_TRY(h, cudaMalloc(&h->d_err, sizeof(int)));
        DWG_CUDA_TRY(h, cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream));
        if (is_device_ptr(points)) {
            dpts = const_cast<float *>(points);
        } else {
            DWG_CUDA_TRY(h, cudaMalloc(&dpts, total * 3 * sizeof(float)));
            own = true;
            DWG_CUDA_TRY(h, cudaMemcpy(dpts, points, total * 3 * sizeof(float),
                                       cudaMemcpyDefault));
        }
        h->n = total;
        for (int c = 0; c < n_clouds; ++c) {
            dwg_ctx *s = new (std::nothrow) dwg_ctx();
            if (!s) return DWG_ERR_OOM;
            h->clouds.push_back(s);
            int rc = create_impl(s, dpts + 3 * off[c], off[c + 1] - off[c]);
            if (rc) return fail(h, rc, "cloud " + std::to_string(c) + ": " + s->err);
            s->depth = auto_depth(s->n);
            s->seed = h->seed + (uint64_t)c;
        }
        return DWG_OK;
    };
    int rc = body();
    if (own) cudaFree(dpts);
    if (rc) {
        set_global_error("dwg_create_batch: " + h->err);
        dwg_destroy(h);
        return rc;
    }
    *out = h;
    return DWG_OK;
}

int dwg_orient_batch(dwg_handle h, float *normals_out, int *iters_out)
{
    if (!h) return DWG_ERR_INVALID;
    if (!h->is_batch) return fail(h, DWG_ERR_STATE, "not a batch handle");
    cudaSetDevice(h->device);
    int rc = batch_prepare(h);
    if (rc) return rc;
    if ((!h->graph_valid || h->graph_gen != batch_gen(h)) && (rc = batch_build_graph(h)))
        return rc;
    cudaEvent_t e0, e1;
    DWG_CUDA_TRY(h, cudaEventCreate(&e0));
    DWG_CUDA_TRY(h, cudaEventCreate(&e1));
    cudaEventRecord(e0, h->stream);
    cudaError_t e = cudaGraphLaunch(h->graph_exec, h->stream);
    cudaEventRecord(e1, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return fail(h, DWG_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(e));
    if ((rc = check_device_err(h))) return rc;
    bool all = true;
    double inter = 0.0;
    int maxit = 0;
    for (size_t c = 0; c < h->clouds.size(); ++c) {
        dwg_ctx *s = h->clouds[c];
        IterState st;
        if ((rc = read_state(s, &st))) return fail(h, rc, s->err);
        if ((rc = check_device_err(s))) return fail(h, rc, s->err);
        int it = std::min(st.iter, s->max_iters);
        if (iters_out) iters_out[c] = it;
        all = all && st.done;
        maxit = std::max(maxit, it);
        double per = (double)s->n * (double)s->n +
                     (s->mode == DWG_UPDATE_LEVELSET ? (double)s->ncorners * (double)s->n : 0.0);
        if (use_tree(s)) {
            unsigned long long cnt = 0;
            DWG_CUDA_TRY(h, cudaMemcpy(&cnt, s->d_counter, sizeof(cnt), cudaMemcpyDeviceToHost));
            inter += (double)cnt;
        } else {
            inter += per * it;
        }
        if (normals_out && (rc = dwg_get_normals(s, normals_out + 3 * h->offsets[c])))
            return fail(h, rc, s->err);
    }
    h->stats.iters = maxit;
    h->stats.converged = all;
    h->stats.interactions = inter;
    h->stats.ms_orient = ms;
    return all ? DWG_OK : DWG_NOT_CONVERGED;
}

}  // extern "C"
