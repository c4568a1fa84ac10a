// dwg_tree.cu -- Barnes-Hut far field for large clouds (paper Sec. 5.2,
// "Octree Traversal").
//
// Hierarchy: the complete binary tree over buckets of kBucket Morton-
// consecutive points that the kNN search also uses (node 1 is the root, node
// k has children 2k, 2k+1, the 2^L leaves are the buckets).  Every node is a
// contiguous Morton range -- an octree node refined at bucket granularity.
//
// Per node, once per cloud (positions are fixed), in double precision with
// separately rounded operations: A = sum a, c = sum a p / A (area-weighted
// mass centre), r = largest point distance from c for a leaf, and for an
// internal node max over its non-empty children of |c_child - c| + r_child.
// Per iteration: M = sum a n (the node's area-weighted normal), leaves
// summed in Morton order, internal nodes as left + right.
//
// Traversal: a warp owns 32 consecutive (Morton-ordered) queries and walks the
// tree once for all of them.  Each stack entry carries the mask of lanes for
// which the node is still open.  A lane uses the node as one dipole (c, M)
// when |q - c|^2 > (beta r)^2 (tested in float32), else the node opens for
// it; a leaf that is open for some lanes is summed exactly by those lanes.
// All lanes read the same node and point records, so the loads are
// broadcasts.  Sums are FP32 terms folded into (hi, lo) two-sum pairs (the
// near field is compensated) and written as chunk-0 partials, so the point
// and corner reduce kernels of the all-pairs path finish the job unchanged.
#include "dwg_internal.cuh"

namespace dwg {

// ---------------------------------------------------------------------------
// build (once per cloud)
// ---------------------------------------------------------------------------
__global__ void k_tree_leaf_sums(const float4 *__restrict__ p4, int64_t n, int64_t nleaf,
                                 double *A, double *Sp)
{
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nleaf) return;
    int64_t node = nleaf + b, j0 = b * kBucket, j1 = min(j0 + kBucket, n);
    double sa = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
    for (int64_t j = j0; j < j1; ++j) {
        float4 p = p4[j];
        double a = (double)p.w;
        sa = __dadd_rn(sa, a);
        sx = __dadd_rn(sx, __dmul_rn(a, (double)p.x));
        sy = __dadd_rn(sy, __dmul_rn(a, (double)p.y));
        sz = __dadd_rn(sz, __dmul_rn(a, (double)p.z));
    }
    A[node] = sa;
    Sp[3 * node] = sx;
    Sp[3 * node + 1] = sy;
    Sp[3 * node + 2] = sz;
}

__global__ void k_tree_level_sums(int64_t first, double *A, double *Sp)
{
    int64_t node = first + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= 2 * first) return;
    int64_t l = 2 * node, r = l + 1;
    A[node] = __dadd_rn(A[l], A[r]);
    for (int k = 0; k < 3; ++k) Sp[3 * node + k] = __dadd_rn(Sp[3 * l + k], Sp[3 * r + k]);
}

__global__ void k_tree_centres(int64_t nn, const double *A, const double *Sp, double *C)
{
    int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (node < 1 || node >= nn) return;
    double a = A[node];
    for (int k = 0; k < 3; ++k) C[3 * node + k] = a > 0.0 ? __ddiv_rn(Sp[3 * node + k], a) : 0.0;
}

__device__ __forceinline__ double dist3(double x, double y, double z)
{
    return __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z)));
}

__global__ void k_tree_leaf_radius(const float4 *__restrict__ p4, int64_t n, int64_t nleaf,
                                   const double *C, double *R)
{
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nleaf) return;
    int64_t node = nleaf + b, j0 = b * kBucket, j1 = min(j0 + kBucket, n);
    double rm = 0.0;
    for (int64_t j = j0; j < j1; ++j) {
        float4 p = p4[j];
        double d = dist3(__dsub_rn((double)p.x, C[3 * node]), __dsub_rn((double)p.y, C[3 * node + 1]),
                         __dsub_rn((double)p.z, C[3 * node + 2]));
        if (d > rm) rm = d;
    }
    R[node] = rm;
}

__global__ void k_tree_level_radius(int64_t first, const double *A, const double *C, double *R)
{
    int64_t node = first + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= 2 * first) return;
    double rm = 0.0;
    for (int64_t ch = 2 * node; ch <= 2 * node + 1; ++ch) {
        if (!(A[ch] > 0.0)) continue;
        double d = __dadd_rn(dist3(__dsub_rn(C[3 * ch], C[3 * node]),
                                   __dsub_rn(C[3 * ch + 1], C[3 * node + 1]),
                                   __dsub_rn(C[3 * ch + 2], C[3 * node + 2])),
                             R[ch]);
        if (d > rm) rm = d;
    }
    R[node] = rm;
}

// traversal record (c_f, (beta r)^2 as float; -1 marks an empty node)
__global__ void k_tree_records(int64_t nn, const double *A, const double *C, const double *R,
                               double beta, float4 *rec)
{
    int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= nn) return;
    if (node < 1 || !(A[node] > 0.0)) {
        rec[node] = make_float4(0.f, 0.f, 0.f, -1.f);
        return;
    }
    double br = __dmul_rn(beta, R[node]);
    rec[node] = make_float4((float)C[3 * node], (float)C[3 * node + 1], (float)C[3 * node + 2],
                            (float)__dmul_rn(br, br));
}

// ---------------------------------------------------------------------------
// moments (per iteration): M = sum a n, then m = M / (4 pi) as float
// ---------------------------------------------------------------------------
__global__ void k_tree_leaf_moments(const float4 *__restrict__ p4, const float4 *__restrict__ nrm,
                                    int64_t n, int64_t nleaf, double *M)
{
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nleaf) return;
    int64_t node = nleaf + b, j0 = b * kBucket, j1 = min(j0 + kBucket, n);
    double mx = 0.0, my = 0.0, mz = 0.0;
    for (int64_t j = j0; j < j1; ++j) {
        double a = (double)p4[j].w;
        float4 v = nrm[j];
        mx = __dadd_rn(mx, __dmul_rn(a, (double)v.x));
        my = __dadd_rn(my, __dmul_rn(a, (double)v.y));
        mz = __dadd_rn(mz, __dmul_rn(a, (double)v.z));
    }
    M[3 * node] = mx;
    M[3 * node + 1] = my;
    M[3 * node + 2] = mz;
}

__global__ void k_tree_level_moments(int64_t first, double *M)
{
    int64_t node = first + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= 2 * first) return;
    int64_t l = 2 * node, r = l + 1;
    for (int k = 0; k < 3; ++k) M[3 * node + k] = __dadd_rn(M[3 * l + k], M[3 * r + k]);
}

__global__ void k_tree_moment_records(int64_t nn, const double *M, float4 *mrec)
{
    int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= nn) return;
    const double fpi = 4.0 * kPi;
    mrec[node] = make_float4((float)__ddiv_rn(M[3 * node], fpi), (float)__ddiv_rn(M[3 * node + 1], fpi),
                             (float)__ddiv_rn(M[3 * node + 2], fpi), 0.f);
}

// ---------------------------------------------------------------------------
// traversal
// ---------------------------------------------------------------------------
__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ void two_sum_f(float &hi, float &lo, float t)
{
    float s = __fadd_rn(hi, t);
    float bb = __fsub_rn(s, hi);
    float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(t, bb));
    lo = __fadd_rn(lo, e);
    hi = s;
}

struct TreeAcc {
    float tw, t1x, t1y, t1z, t2x, t2y, t2z;  // current batch (plain FP32)
    float hw, lw, hgx, lgx, hgy, lgy, hgz, lgz;
    int pending;
};

template <bool GRAD, bool SCREENED>
__device__ __forceinline__ void tree_term(TreeAcc &A, float qx, float qy, float qz, float px,
                                          float py, float pz, float mx, float my, float mz,
                                          const EvalParams &ep)
{
    float dx = px - qx, dy = py - qy, dz = pz - qz;
    float rr = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, ep.eps2)));
    float inv = rsqrt_approx(rr);
    float md = fmaf(mz, dz, fmaf(my, dy, mx * dx));
    float i2 = inv * inv, i3 = i2 * inv;
    if (!SCREENED) {
        float phi = md * i3;
        A.tw += phi;
        if (GRAD) {
            float c = phi * i2;
            A.t1x = fmaf(c, dx, A.t1x); A.t1y = fmaf(c, dy, A.t1y); A.t1z = fmaf(c, dz, A.t1z);
            A.t2x = fmaf(mx, i3, A.t2x); A.t2y = fmaf(my, i3, A.t2y); A.t2z = fmaf(mz, i3, A.t2z);
        }
    } else {
        float rho = rr * inv;
        float e = ex2_approx(rho * ep.nl2e_s);
        float F = fmaf(e, rho * ep.s, e);
        float phi = md * i3;
        A.tw = fmaf(F, phi, A.tw);
        if (GRAD) {
            float fi3 = F * i3;
            float cc = fmaf(3.f, F * i2, ep.s2 * e);
            float c = phi * cc;
            A.t1x = fmaf(c, dx, A.t1x); A.t1y = fmaf(c, dy, A.t1y); A.t1z = fmaf(c, dz, A.t1z);
            A.t2x = fmaf(mx, fi3, A.t2x); A.t2y = fmaf(my, fi3, A.t2y); A.t2z = fmaf(mz, fi3, A.t2z);
        }
    }
    A.pending++;
}

template <bool GRAD, bool SCREENED>
__device__ __forceinline__ void tree_fold(TreeAcc &A)
{
    two_sum_f(A.hw, A.lw, A.tw);
    if (GRAD) {
        float gx = SCREENED ? A.t1x - A.t2x : fmaf(3.f, A.t1x, -A.t2x);
        float gy = SCREENED ? A.t1y - A.t2y : fmaf(3.f, A.t1y, -A.t2y);
        float gz = SCREENED ? A.t1z - A.t2z : fmaf(3.f, A.t1z, -A.t2z);
        two_sum_f(A.hgx, A.lgx, gx);
        two_sum_f(A.hgy, A.lgy, gy);
        two_sum_f(A.hgz, A.lgz, gz);
    }
    A.tw = A.t1x = A.t1y = A.t1z = A.t2x = A.t2y = A.t2z = 0.f;
    A.pending = 0;
}

constexpr int kTreeThreads = 128;
constexpr int kTreeStack = 64;

template <bool GRAD, bool SCREENED>
__global__ void __launch_bounds__(kTreeThreads)
    k_tree_gwn(const float4 *__restrict__ q, int64_t m, const float4 *__restrict__ rec,
               const float4 *__restrict__ mrec, const float *__restrict__ src, int64_t n,
               int levels, EvalParams ep, float *__restrict__ part, int64_t stride,
               unsigned long long *__restrict__ counter, int *err, const IterState *st)
{
    if (st && cloud_idle(st)) return;  // finished cloud of a batch
    __shared__ int s_node[kTreeThreads / 32][kTreeStack];
    __shared__ unsigned s_mask[kTreeThreads / 32][kTreeStack];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * kTreeThreads + threadIdx.x;
    const bool valid = i < m;
    const float4 qq = q[valid ? i : m - 1];
    const unsigned lanebit = 1u << lane;
    const int64_t nleaf = (int64_t)1 << levels;
    TreeAcc A = {};
    unsigned long long evals = 0;
    int sp = 0;
    if (lane == 0) {
        s_node[wid][0] = 1;
        s_mask[wid][0] = __ballot_sync(0xffffffffu, valid);
    } else {
        __ballot_sync(0xffffffffu, valid);
    }
    sp = 1;
    __syncwarp();
    while (sp > 0) {
        --sp;
        const int node = s_node[wid][sp];
        const unsigned mask = s_mask[wid][sp];
        __syncwarp();
        const float4 cr = rec[node];
        if (cr.w < 0.f) continue;  // empty node
        const bool active = (mask & lanebit) != 0;
        float dx = __fsub_rn(qq.x, cr.x), dy = __fsub_rn(qq.y, cr.y), dz = __fsub_rn(qq.z, cr.z);
        float d2 = fmaf(dz, dz, fmaf(dy, dy, __fmul_rn(dx, dx)));
        const bool far = active && d2 > cr.w;
        if (far) {
            float4 mm = mrec[node];
            tree_term<GRAD, SCREENED>(A, qq.x, qq.y, qq.z, cr.x, cr.y, cr.z, mm.x, mm.y, mm.z, ep);
            ++evals;
        }
        const unsigned near = __ballot_sync(0xffffffffu, active && !far);
        if (near) {
            if (node >= nleaf) {
                int64_t j0 = (int64_t)(node - nleaf) * kBucket, j1 = min(j0 + kBucket, n);
                if (near & lanebit) {
                    for (int64_t j = j0; j < j1; ++j) {
                        const float *r = src + j * kSrcFloats;
                        tree_term<GRAD, SCREENED>(A, qq.x, qq.y, qq.z, r[0], r[2], r[4], r[6],
                                                  r[8], r[10], ep);
                    }
                    evals += (unsigned long long)(j1 - j0);
                }
            } else {
                if (sp + 2 > kTreeStack) {
                    if (lane == 0) atomicOr(err, kErrStack);
                    break;
                }
                if (lane == 0) {
                    s_node[wid][sp] = 2 * node + 1;
                    s_mask[wid][sp] = near;
                    s_node[wid][sp + 1] = 2 * node;
                    s_mask[wid][sp + 1] = near;
                }
                sp += 2;
                __syncwarp();
            }
        }
        if (A.pending >= 16) tree_fold<GRAD, SCREENED>(A);
    }
    tree_fold<GRAD, SCREENED>(A);
    if (valid) {
        part[0 * stride + i] = A.hw;
        part[1 * stride + i] = A.lw;
        if (GRAD) {
            part[2 * stride + i] = A.hgx;
            part[3 * stride + i] = A.lgx;
            part[4 * stride + i] = A.hgy;
            part[5 * stride + i] = A.lgy;
            part[6 * stride + i] = A.hgz;
            part[7 * stride + i] = A.lgz;
        }
    }
    // evaluations performed (for the throughput metric)
    for (int o = 16; o > 0; o >>= 1) evals += __shfl_xor_sync(0xffffffffu, evals, o);
    if (lane == 0 && counter) atomicAdd(counter, evals);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
int build_tree(Ctx *c)
{
    if (c->tree_built) return DWG_OK;
    const int64_t nleaf = (int64_t)1 << c->knn_levels, nn = 2 * nleaf;
    const int B = 256;
    DWG_CUDA_TRY(c, cudaMalloc(&c->d_tree_A, nn * sizeof(double)));
    DWG_CUDA_TRY(c, cudaMalloc(&c->d_tree_C, 3 * nn * sizeof(double)));
    DWG_CUDA_TRY(c, cudaMalloc(&c->d_tree_R, nn * sizeof(double)));
    DWG_CUDA_TRY(c, cudaMalloc(&c->d_tree_M, 3 * nn * sizeof(double)));
    DWG_CUDA_TRY(c, cudaMalloc(&c->d_tree_rec, nn * sizeof(float4)));
    DWG_CUDA_TRY(c, cudaMalloc(&c->d_tree_mrec, nn * sizeof(float4)));
    DWG_CUDA_TRY(c, cudaMemsetAsync(c->d_tree_A, 0, nn * sizeof(double), c->stream));
    DWG_CUDA_TRY(c, cudaMemsetAsync(c->d_tree_M, 0, 3 * nn * sizeof(double), c->stream));
    double *Sp = nullptr;
    DWG_CUDA_TRY(c, cudaMalloc(&Sp, 3 * nn * sizeof(double)));
    k_tree_leaf_sums<<<(unsigned)ceil_div(nleaf, B), B, 0, c->stream>>>(c->d_p4, c->n, nleaf,
                                                                         c->d_tree_A, Sp);
    for (int lv = c->knn_levels - 1; lv >= 0; --lv) {
        int64_t first = (int64_t)1 << lv;
        k_tree_level_sums<<<(unsigned)ceil_div(first, B), B, 0, c->stream>>>(first, c->d_tree_A, Sp);
    }
    k_tree_centres<<<(unsigned)ceil_div(nn, B), B, 0, c->stream>>>(nn, c->d_tree_A, Sp, c->d_tree_C);
    k_tree_leaf_radius<<<(unsigned)ceil_div(nleaf, B), B, 0, c->stream>>>(c->d_p4, c->n, nleaf,
                                                                           c->d_tree_C, c->d_tree_R);
    for (int lv = c->knn_levels - 1; lv >= 0; --lv) {
        int64_t first = (int64_t)1 << lv;
        k_tree_level_radius<<<(unsigned)ceil_div(first, B), B, 0, c->stream>>>(
            first, c->d_tree_A, c->d_tree_C, c->d_tree_R);
    }
    DWG_CUDA_TRY(c, cudaGetLastError());
    DWG_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    cudaFree(Sp);
    c->tree_built = true;
    c->tree_beta_set = -1.0;
    return DWG_OK;
}

int tree_records(Ctx *c)
{
    if (c->tree_beta_set == (double)c->tree_beta) return DWG_OK;
    const int64_t nn = (int64_t)2 << c->knn_levels;
    k_tree_records<<<(unsigned)ceil_div(nn, 256), 256, 0, c->stream>>>(
        nn, c->d_tree_A, c->d_tree_C, c->d_tree_R, (double)c->tree_beta, c->d_tree_rec);
    DWG_CUDA_TRY(c, cudaGetLastError());
    c->tree_beta_set = (double)c->tree_beta;
    return DWG_OK;
}

cudaError_t launch_tree_moments(Ctx *c)
{
    const int64_t nleaf = (int64_t)1 << c->knn_levels, nn = 2 * nleaf;
    const int B = 256;
    k_tree_leaf_moments<<<(unsigned)ceil_div(nleaf, B), B, 0, c->stream>>>(c->d_p4, c->d_nrm, c->n,
                                                                            nleaf, c->d_tree_M);
    for (int lv = c->knn_levels - 1; lv >= 0; --lv) {
        int64_t first = (int64_t)1 << lv;
        k_tree_level_moments<<<(unsigned)ceil_div(first, B), B, 0, c->stream>>>(first, c->d_tree_M);
    }
    k_tree_moment_records<<<(unsigned)ceil_div(nn, B), B, 0, c->stream>>>(nn, c->d_tree_M,
                                                                           c->d_tree_mrec);
    return cudaGetLastError();
}

cudaError_t launch_tree_gwn(Ctx *c, const float4 *q, int64_t m, bool grad, float *part,
                            int64_t stride, const IterState *st)
{
    EvalParams ep = make_eval_params(c);
    unsigned blocks = (unsigned)ceil_div(m, kTreeThreads);
    if (grad) {
        if (ep.screened)
            k_tree_gwn<true, true><<<blocks, kTreeThreads, 0, c->stream>>>(
                q, m, c->d_tree_rec, c->d_tree_mrec, c->d_src, c->n, c->knn_levels, ep, part, stride,
                c->d_counter, c->d_err, st);
        else
            k_tree_gwn<true, false><<<blocks, kTreeThreads, 0, c->stream>>>(
                q, m, c->d_tree_rec, c->d_tree_mrec, c->d_src, c->n, c->knn_levels, ep, part, stride,
                c->d_counter, c->d_err, st);
    } else {
        if (ep.screened)
            k_tree_gwn<false, true><<<blocks, kTreeThreads, 0, c->stream>>>(
                q, m, c->d_tree_rec, c->d_tree_mrec, c->d_src, c->n, c->knn_levels, ep, part, stride,
                c->d_counter, c->d_err, st);
        else
            k_tree_gwn<false, false><<<blocks, kTreeThreads, 0, c->stream>>>(
                q, m, c->d_tree_rec, c->d_tree_mrec, c->d_src, c->n, c->knn_levels, ep, part, stride,
                c->d_counter, c->d_err, st);
    }
    return cudaGetLastError();
}

}  // namespace dwg
