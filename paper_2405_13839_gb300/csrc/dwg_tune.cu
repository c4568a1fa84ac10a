// dwg_tune.cu -- the autotuner (a project extension; the paper fixes its
// parameters by hand, Sec. 5.1 and Sec. 5.2).
//
// For one handle's cloud it chooses, by measurement on the handle's stream:
//   - the evaluator shape (query pairs per thread, CTA size) of the exact
//     all-pairs sums, separately for w and grad w at the points and for w at
//     the octree-leaf corners: every compiled shape is launched on the real
//     sources and timed with CUDA events (median of three after a warm-up);
//   - for the Barnes-Hut path, the leaf size, the form of the opening test
//     (per query, or per 64-query group) and the opening angle: for each leaf
//     size and form the largest opening angle whose w stays within the
//     caller's error budget on a sample of the queries (against the exact
//     all-pairs sum of the same sample), then the fastest of these by timing
//     a full evaluation at the points and the corners;
//   - for DWG_PATH_AUTO, the faster of the two paths (the tree only when it
//     meets the budget).
// Results are appended to a cache file (one JSON object per line, keyed by
// the GPU's name and SM count and the problem: sizes, kernel, update rule,
// requested path, budget), which later calls read instead of measuring.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <string>
#include <vector>

#include "dwg_internal.cuh"

namespace dwg {

namespace {

constexpr float kThetas[] = {0.9f, 0.8f, 0.7f, 0.6f, 0.5f, 0.4f, 0.3f, 0.2f};
constexpr int kLeaves[] = {16, 32, 64, 128};
constexpr int64_t kSampleEach = 2048;        // tree-accuracy sample: points and corners
constexpr double kMaxTimedInteractions = 4e11;  // cap of one timed all-pairs launch

// sample of `count` queries out of m: runs of 64 consecutive ones (a warp
// group of the group traversal sees its real bounding boxes) spread evenly
__global__ void k_sample_runs(const float4 *__restrict__ src, int64_t m, int64_t count,
                              float4 *__restrict__ dst)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int64_t runs = (count + 63) / 64;
    const int64_t step = max((int64_t)64, m / runs);
    const int64_t j = (i / 64) * step + (i % 64);
    dst[i] = src[min(j, m - 1)];
}

__global__ void k_max_abs_diff(const float *__restrict__ a, const float *__restrict__ b, int64_t m,
                               float *out)
{
    __shared__ float sh[256];
    float v = 0.f;
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
        float d = fabsf(a[i] - b[i]);
        if (!(d <= v)) v = d;  // NaN propagates as the maximum
    }
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            float u = sh[threadIdx.x + o];
            if (!(u <= sh[threadIdx.x])) sh[threadIdx.x] = u;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

struct Buf {
    void *p = nullptr;
    ~Buf() { cudaFree(p); }
    template <class T>
    T *as() { return (T *)p; }
};

#define TUNE_TRY(call)                                                       \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess) {                                             \
            c->err = std::string("autotune: ") + #call + ": " + cudaGetErrorString(e_); \
            return e_ == cudaErrorMemoryAllocation ? DWG_ERR_OOM : DWG_ERR_CUDA; \
        }                                                                    \
    } while (0)

// median device time of `launch` over 3 runs after one warm-up
int time_ms(Ctx *c, const std::function<int()> &launch, double *ms_out)
{
    cudaEvent_t e0, e1;
    TUNE_TRY(cudaEventCreate(&e0));
    TUNE_TRY(cudaEventCreate(&e1));
    int rc = launch();
    std::vector<float> t;
    for (int r = 0; r < 3 && !rc; ++r) {
        cudaEventRecord(e0, c->stream);
        rc = launch();
        cudaEventRecord(e1, c->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = DWG_ERR_CUDA;
            c->err = "autotune: timing failed";
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        t.push_back(ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    std::sort(t.begin(), t.end());
    *ms_out = t[t.size() / 2];
    return DWG_OK;
}

int device_error(Ctx *c)
{
    int herr = 0;
    TUNE_TRY(cudaMemcpyAsync(&herr, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    TUNE_TRY(cudaStreamSynchronize(c->stream));
    if (herr) {
        cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
        c->err = "autotune: a device-side check failed during the measurements";
        return (herr & kErrTimeout) ? DWG_ERR_TIMEOUT : DWG_ERR_CUDA;
    }
    return DWG_OK;
}

// fastest evaluator variant for m queries (a prefix of q, capped so that one
// launch stays below kMaxTimedInteractions); ms scaled to all m queries
int tune_shape(Ctx *c, const float4 *q, int64_t m, bool grad, int *best_v, double *best_ms)
{
    int64_t mt = m;
    if ((double)mt * (double)c->n > kMaxTimedInteractions)
        mt = std::max<int64_t>(4096, (int64_t)(kMaxTimedInteractions / (double)c->n));
    mt = std::min(mt, m);
    const int nv = eval_variant_count(grad);
    int maxch = 1;
    for (int v = 0; v < nv; ++v) maxch = std::max(maxch, eval_chunks_variant(c, mt, grad, v));
    Buf part;
    TUNE_TRY(cudaMalloc(&part.p, (size_t)maxch * (grad ? 8 : 2) * mt * sizeof(float)));
    *best_v = -1;
    *best_ms = 0.0;
    for (int v = 0; v < nv; ++v) {
        const int nch = eval_chunks_variant(c, mt, grad, v);
        double ms = 0.0;
        int rc = time_ms(c, [&]() {
            return eval_launch_variant(c, q, mt, grad, v, nch, part.as<float>(), mt);
        }, &ms);
        if (rc) return rc;
        ms *= (double)m / (double)mt;
        if (*best_v < 0 || ms < *best_ms) {
            *best_v = v;
            *best_ms = ms;
        }
    }
    return device_error(c);
}

// w at the sample queries by the tree path (current leaf size and beta)
int tree_w(Ctx *c, const float4 *q, int64_t m, float *part, float *w)
{
    int rc = tree_records(c);
    if (rc) return rc;
    if (launch_tree_moments(c) != cudaSuccess ||
        launch_tree_gwn(c, q, m, false, part, m, nullptr) != cudaSuccess ||
        launch_reduce_w(c, part, 1, m, w) != cudaSuccess) {
        c->err = "autotune: tree launch failed";
        return DWG_ERR_CUDA;
    }
    return DWG_OK;
}

std::string key_of(const Ctx *c, int path_req, double budget)
{
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, c->device) != cudaSuccess) prop.name[0] = 0;
    char buf[512];
    snprintf(buf, sizeof buf,
             "\"gpu\": \"%s\", \"sms\": %d, \"n\": %lld, \"corners\": %lld, \"kernel\": %d, "
             "\"screening\": %.9g, \"mode\": %d, \"path_request\": %d, \"budget\": %.9g",
             prop.name, prop.multiProcessorCount, (long long)c->n,
             (long long)(c->mode == DWG_UPDATE_LEVELSET ? c->ncorners : 0), c->kernel,
             (double)(c->kernel == DWG_KERNEL_SCREENED ? c->lambda : 0.f), c->mode, path_req,
             budget);
    return buf;
}

bool json_num(const std::string &line, const char *name, double *v)
{
    std::string pat = std::string("\"") + name + "\": ";
    size_t p = line.find(pat);
    if (p == std::string::npos) return false;
    return sscanf(line.c_str() + p + pat.size(), "%lf", v) == 1;
}

bool cache_lookup(const char *path, const std::string &key, dwg_tuning *t)
{
    if (!path) return false;
    FILE *f = fopen(path, "r");
    if (!f) return false;
    bool found = false;
    std::string line;
    char chunk[1024];
    while (fgets(chunk, sizeof chunk, f)) {
        line += chunk;
        if (line.empty() || line.back() != '\n') continue;
        if (line.find(key) != std::string::npos) {
            double v[11];
            const char *names[] = {"path", "points_pairs", "points_threads", "corners_pairs",
                                   "corners_threads", "tree_leaf", "theta", "w_err", "ms_points",
                                   "ms_corners", "tree_group"};
            bool ok = true;
            for (int k = 0; k < 11; ++k) ok = ok && json_num(line, names[k], &v[k]);
            if (ok) {
                t->path = (int)v[0];
                t->points_pairs = (int)v[1];
                t->points_threads = (int)v[2];
                t->corners_pairs = (int)v[3];
                t->corners_threads = (int)v[4];
                t->tree_leaf = (int)v[5];
                t->theta = (float)v[6];
                t->w_err = v[7];
                t->ms_points = v[8];
                t->ms_corners = v[9];
                t->tree_group = (int)v[10];
                found = true;  // the last matching line wins
            }
        }
        line.clear();
    }
    fclose(f);
    return found;
}

void cache_store(const char *path, const std::string &key, const dwg_tuning &t)
{
    if (!path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f,
            "{%s, \"path\": %d, \"points_pairs\": %d, \"points_threads\": %d, "
            "\"corners_pairs\": %d, \"corners_threads\": %d, \"tree_leaf\": %d, \"theta\": %.9g, "
            "\"w_err\": %.9g, \"ms_points\": %.9g, \"ms_corners\": %.9g, \"tree_group\": %d}\n",
            key.c_str(), t.path, t.points_pairs, t.points_threads, t.corners_pairs,
            t.corners_threads, t.tree_leaf, (double)t.theta, t.w_err, t.ms_points, t.ms_corners,
            t.tree_group);
    fclose(f);
}

int variant_of(bool grad, int pairs, int threads)
{
    for (int v = 0; v < eval_variant_count(grad); ++v) {
        int p, nt;
        eval_variant_shape(grad, v, &p, &nt);
        if (p == pairs && nt == threads) return v;
    }
    return -1;
}

}  // namespace

void tuning_of(const Ctx *c, dwg_tuning *t)
{
    memset(t, 0, sizeof *t);
    t->path = use_tree(c) ? DWG_PATH_TREE : DWG_PATH_ALLPAIRS;
    eval_variant_shape(true, c->var_grad, &t->points_pairs, &t->points_threads);
    eval_variant_shape(false, c->var_w, &t->corners_pairs, &t->corners_threads);
    t->tree_leaf = c->tree_leaf;
    t->theta = 1.0f / c->tree_beta;
    t->tree_group = c->tree_group;
    t->knn_lists = c->knn_lists;
    t->w_err = c->tune_w_err;
    t->ms_points = c->tune_ms_points;
    t->ms_corners = c->tune_ms_corners;
}

int apply_tuning(Ctx *c, const dwg_tuning *t)
{
    if (t->path != DWG_PATH_ALLPAIRS && t->path != DWG_PATH_TREE) {
        c->err = "tuning: path must be DWG_PATH_ALLPAIRS or DWG_PATH_TREE";
        return DWG_ERR_INVALID;
    }
    int vg = variant_of(true, t->points_pairs, t->points_threads);
    int vw = variant_of(false, t->corners_pairs, t->corners_threads);
    if (vg < 0 || vw < 0) {
        c->err = "tuning: no compiled evaluator has this (pairs, threads) shape";
        return DWG_ERR_INVALID;
    }
    bool leaf_ok = false;
    for (int L : kLeaves) leaf_ok = leaf_ok || L == t->tree_leaf;
    if (!leaf_ok) {
        c->err = "tuning: tree_leaf must be 16, 32, 64 or 128";
        return DWG_ERR_INVALID;
    }
    if (!(t->theta > 0.f) || !(t->theta <= 1.f)) {
        c->err = "tuning: theta must be in (0, 1]";
        return DWG_ERR_INVALID;
    }
    if (t->tree_group != 0 && t->tree_group != 1) {
        c->err = "tuning: tree_group must be 0 or 1";
        return DWG_ERR_INVALID;
    }
    if (t->knn_lists != 0 && t->knn_lists != 1) {
        c->err = "tuning: knn_lists must be 0 or 1";
        return DWG_ERR_INVALID;
    }
    c->tree_group = t->tree_group;
    c->knn_lists = t->knn_lists;
    c->path = t->path;
    c->var_grad = vg;
    c->var_w = vw;
    if (c->tree_leaf != t->tree_leaf) {
        c->tree_leaf = t->tree_leaf;
        c->tree_built = false;
    }
    c->tree_beta = 1.0f / t->theta;
    c->tune_w_err = t->w_err;
    c->tune_ms_points = t->ms_points;
    c->tune_ms_corners = t->ms_corners;
    ++c->bufgen;
    return DWG_OK;
}

// The winding number's scale inside a closed surface, 1 / (mean area per
// point) x mean a: the area per point estimated from the spacing, pi r^2 / 10
// with r the median distance to the 10th nearest other point (a disc of
// radius r around a point of a surface sampling holds about 10 others).
int w_scale(Ctx *c, double *scale)
{
    const int64_t m = std::min<int64_t>(2048, c->n);
    Buf d, a;
    TUNE_TRY(cudaMalloc(&d.p, m * sizeof(float)));
    TUNE_TRY(launch_spacing(c, m, d.as<float>()));
    std::vector<float> h(m);
    std::vector<float4> p4(c->n < 65536 ? c->n : 65536);
    TUNE_TRY(cudaMemcpyAsync(h.data(), d.p, m * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    TUNE_TRY(cudaMemcpyAsync(p4.data(), c->d_p4, p4.size() * sizeof(float4), cudaMemcpyDeviceToHost,
                             c->stream));
    TUNE_TRY(cudaStreamSynchronize(c->stream));
    std::sort(h.begin(), h.end());
    const double r = h[m / 2];
    double abar = 0.0;
    for (const float4 &v : p4) abar += (double)v.w;
    abar /= (double)p4.size();
    const double area_per_point = kPi * r * r / 10.0;
    *scale = area_per_point > 0.0 ? abar / area_per_point : 1.0;
    return DWG_OK;
}

int autotune(Ctx *c, int what, double budget, const char *cache_path, dwg_tuning *out)
{
    if (!(budget > 0.0) && (what & DWG_TUNE_TREE)) {
        c->err = "autotune: the error budget must be > 0";
        return DWG_ERR_INVALID;
    }
    const int path_req = c->path;
    int rc = engine_prepare(c);
    if (rc) return rc;
    if (what & DWG_TUNE_RELATIVE) {
        double scale = 1.0;
        if ((rc = w_scale(c, &scale))) return rc;
        budget *= scale;
    }
    const std::string key = key_of(c, path_req, budget) + ", \"what\": " + std::to_string(what);
    dwg_tuning t;
    tuning_of(c, &t);  // fields the cache does not hold keep the handle's values
    if (cache_lookup(cache_path, key, &t)) {
        if ((rc = apply_tuning(c, &t))) return rc;
        t.from_cache = 1;
        if (out) *out = t;
        return DWG_OK;
    }
    tuning_of(c, &t);
    const bool lset = c->mode == DWG_UPDATE_LEVELSET;

    // 1. evaluator shapes of the exact path
    double ap_ms_p = 0.0, ap_ms_c = 0.0;
    int vg = c->var_grad, vw = c->var_w;
    const bool want_ap = path_req != DWG_PATH_TREE;
    if ((what & DWG_TUNE_SHAPES) && want_ap) {
        if ((rc = tune_shape(c, c->d_p4, c->n, true, &vg, &ap_ms_p))) return rc;
        if (lset && (rc = tune_shape(c, c->d_corner_pos, c->ncorners, false, &vw, &ap_ms_c)))
            return rc;
        eval_variant_shape(true, vg, &t.points_pairs, &t.points_threads);
        eval_variant_shape(false, vw, &t.corners_pairs, &t.corners_threads);
    }

    // 2. Barnes-Hut leaf size and opening angle within the budget
    bool tree_ok = false;
    double tr_ms_p = 0.0, tr_ms_c = 0.0;
    int best_leaf = c->tree_leaf, best_group = c->tree_group;
    float best_theta = 1.0f / c->tree_beta;
    double best_err = 0.0;
    const bool want_tree = path_req != DWG_PATH_ALLPAIRS && (what & DWG_TUNE_TREE);
    if (want_tree) {
        const int64_t sp = std::min<int64_t>(kSampleEach, c->n);
        const int64_t sc = lset ? std::min<int64_t>(kSampleEach, c->ncorners) : 0;
        const int64_t S = sp + sc;
        Buf q, part, wex, wtr, dmax;
        TUNE_TRY(cudaMalloc(&q.p, S * sizeof(float4)));
        const int nch = eval_chunks_variant(c, S, false, 0);
        TUNE_TRY(cudaMalloc(&part.p, (size_t)std::max(nch, 1) * 2 * S * sizeof(float)));
        TUNE_TRY(cudaMalloc(&wex.p, S * sizeof(float)));
        TUNE_TRY(cudaMalloc(&wtr.p, S * sizeof(float)));
        TUNE_TRY(cudaMalloc(&dmax.p, sizeof(float)));
        k_sample_runs<<<(unsigned)ceil_div(sp, 256), 256, 0, c->stream>>>(c->d_p4, c->n, sp,
                                                                            q.as<float4>());
        if (sc > 0)
            k_sample_runs<<<(unsigned)ceil_div(sc, 256), 256, 0, c->stream>>>(
                c->d_corner_pos, c->ncorners, sc, q.as<float4>() + sp);
        TUNE_TRY(cudaGetLastError());
        // exact reference: all-pairs w of the sample
        if ((rc = eval_launch_variant(c, q.as<float4>(), S, false, 0, nch, part.as<float>(), S)))
            return rc;
        TUNE_TRY(launch_reduce_w(c, part.as<float>(), nch, S, wex.as<float>()));
        const int saved_leaf = c->tree_leaf;
        const float saved_beta = c->tree_beta;
        const int saved_group = c->tree_group;
        for (int L : kLeaves)
        for (int G = 0; G < 2; ++G) {
            if ((int64_t)L > std::max<int64_t>(16, c->n / 4)) break;  // at least 4 leaves
            c->tree_group = G;
            if (c->tree_leaf != L || !c->tree_built) {
                c->tree_leaf = L;
                c->tree_built = false;
                if ((rc = build_tree(c))) return rc;
            }
            float th_ok = -1.f;
            double err_ok = 0.0;
            for (float th : kThetas) {
                c->tree_beta = 1.0f / th;
                if ((rc = tree_w(c, q.as<float4>(), S, part.as<float>(), wtr.as<float>())))
                    return rc;
                k_max_abs_diff<<<1, 256, 0, c->stream>>>(wex.as<float>(), wtr.as<float>(), S,
                                                        dmax.as<float>());
                float e = 0.f;
                TUNE_TRY(cudaMemcpyAsync(&e, dmax.p, sizeof(float), cudaMemcpyDeviceToHost,
                                         c->stream));
                TUNE_TRY(cudaStreamSynchronize(c->stream));
                if (e <= budget) {
                    th_ok = th;
                    err_ok = e;
                    break;  // the largest angle that meets the budget is the cheapest
                }
            }
            if (th_ok < 0.f) continue;
            c->tree_beta = 1.0f / th_ok;
            if ((rc = tree_records(c))) return rc;
            if (G) {  // the iteration evaluates interaction lists, built once
                bool built = false;
                if ((rc = tree_lists(c, c->lists_p, c->d_p4, c->n, &built))) return rc;
                if (lset &&
                    (rc = tree_lists(c, c->lists_c, c->d_corner_pos, c->ncorners, &built)))
                    return rc;
            }
            double mp = 0.0, mc = 0.0;
            rc = time_ms(c, [&]() {
                if (launch_tree_moments(c) != cudaSuccess ||
                    launch_tree_iter(c, c->lists_p, c->d_p4, c->n, true, c->d_part_p, c->n,
                                     nullptr) != cudaSuccess)
                    return DWG_ERR_CUDA;
                return DWG_OK;
            }, &mp);
            if (!rc && lset)
                rc = time_ms(c, [&]() {
                    return launch_tree_iter(c, c->lists_c, c->d_corner_pos, c->ncorners, false,
                                            c->d_part_c, c->ncorners, nullptr) == cudaSuccess
                               ? DWG_OK
                               : DWG_ERR_CUDA;
                }, &mc);
            if (rc) {
                if (c->err.empty()) c->err = "autotune: tree launch failed";
                return rc;
            }
            if (!tree_ok || mp + mc < tr_ms_p + tr_ms_c) {
                tree_ok = true;
                best_leaf = L;
                best_group = G;
                best_theta = th_ok;
                best_err = err_ok;
                tr_ms_p = mp;
                tr_ms_c = mc;
            }
        }
        c->tree_leaf = saved_leaf;
        c->tree_beta = saved_beta;
        c->tree_group = saved_group;
        c->tree_built = false;
        free_lists(c->lists_p);
        free_lists(c->lists_c);
        if ((rc = device_error(c))) return rc;
        if (path_req == DWG_PATH_TREE && !tree_ok) {
            c->err = "autotune: no opening angle down to 0.2 meets the error budget";
            return DWG_ERR_INVALID;
        }
    }
    if (tree_ok) {
        t.tree_leaf = best_leaf;
        t.theta = best_theta;
        t.tree_group = best_group;
    }

    // 3. the path
    if (path_req == DWG_PATH_TREE) {
        t.path = DWG_PATH_TREE;
    } else if (path_req == DWG_PATH_ALLPAIRS) {
        t.path = DWG_PATH_ALLPAIRS;
    } else if (tree_ok && (what & DWG_TUNE_SHAPES)) {
        t.path = (tr_ms_p + tr_ms_c < ap_ms_p + ap_ms_c) ? DWG_PATH_TREE : DWG_PATH_ALLPAIRS;
    } else {
        t.path = use_tree(c) && tree_ok ? DWG_PATH_TREE : DWG_PATH_ALLPAIRS;
    }
    if (t.path == DWG_PATH_TREE) {
        t.w_err = best_err;
        t.ms_points = tr_ms_p;
        t.ms_corners = tr_ms_c;
    } else {
        t.w_err = 0.0;
        t.ms_points = ap_ms_p;
        t.ms_corners = ap_ms_c;
    }
    if ((rc = apply_tuning(c, &t))) return rc;
    cache_store(cache_path, key, t);
    t.from_cache = 0;
    if (out) *out = t;
    return DWG_OK;
}

}  // namespace dwg
