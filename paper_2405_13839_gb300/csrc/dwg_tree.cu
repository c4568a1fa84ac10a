// dwg_tree.cu -- Barnes-Hut far field for large clouds (paper Sec. 5.2,
// "Octree Traversal").
//
// Hierarchy: the complete binary tree over leaves of `tree_leaf` (16, 32, 64
// or 128, a tuning choice) Morton-consecutive points (node 1 is the root,
// node k has children 2k, 2k+1, the 2^L leaves hold the points).  Every node
// is a contiguous Morton range -- an octree node refined at leaf
// granularity.
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
//
// Group traversal (tree_group = 1): the opening test is applied to the
// bounding box of a warp's 64 consecutive queries (two per lane), which is
// conservative -- a node far from the box is far from each of its queries.
// The warp walks the tree 32 nodes at a time (one per lane; ballots and
// prefix counts append to shared-memory lists), collects the far nodes'
// dipole records and the near leaves' point records in shared memory, and
// every lane evaluates the whole list for its two queries with the packed
// f32x2 inner loop of the all-pairs path: no divergence and broadcast reads.
// Each query does a few more terms than under its own test and gets a
// smaller error bound.
#include <string.h>

#include <algorithm>

#include "dwg_internal.cuh"
#include "dwg_packed.cuh"

namespace dwg {

// ---------------------------------------------------------------------------
// build (once per cloud)
// ---------------------------------------------------------------------------
__global__ void k_tree_leaf_sums(const float4 *__restrict__ p4, int64_t n, int64_t nleaf,
                                 int bucket, double *A, double *Sp)
{
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nleaf) return;
    int64_t node = nleaf + b, j0 = b * bucket, j1 = min(j0 + bucket, n);
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
                                   int bucket, const double *C, double *R)
{
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nleaf) return;
    int64_t node = nleaf + b, j0 = b * bucket, j1 = min(j0 + bucket, n);
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

// Largest clamp radius of the modified kernel per node (sqrt of the stored
// float delta^2, in double): leaves over their points, then level by level.
__global__ void k_tree_leaf_dmax(const float *__restrict__ delta2, int64_t n, int64_t nleaf,
                                 int bucket, double *Dmax)
{
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nleaf) return;
    int64_t j0 = b * bucket, j1 = min(j0 + bucket, n);
    double dm = 0.0;
    for (int64_t j = j0; j < j1; ++j) dm = fmax(dm, sqrt((double)delta2[j]));
    Dmax[nleaf + b] = dm;
}

__global__ void k_tree_level_dmax(int64_t first, double *Dmax)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= first) return;
    int64_t node = first + t;
    Dmax[node] = fmax(Dmax[2 * node], Dmax[2 * node + 1]);
}

// traversal record (c_f, (beta r)^2 as float; -1 marks an empty node).  With
// the modified kernel's radii (Dmax non-null) the opening radius is
// max(beta r, r + Dmax): a far node then never holds a point whose radius
// reaches the query, and its dipole is the unclamped one.
__global__ void k_tree_records(int64_t nn, const double *A, const double *C, const double *R,
                               double beta, const double *Dmax, float4 *rec)
{
    int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= nn) return;
    if (node < 1 || !(A[node] > 0.0)) {
        rec[node] = make_float4(0.f, 0.f, 0.f, -1.f);
        return;
    }
    double br = __dmul_rn(beta, R[node]);
    if (Dmax) br = fmax(br, __dadd_rn(R[node], Dmax[node]));
    rec[node] = make_float4((float)C[3 * node], (float)C[3 * node + 1], (float)C[3 * node + 2],
                            (float)__dmul_rn(br, br));
}

// ---------------------------------------------------------------------------
// moments (per iteration): M = sum a n, then m = M / (4 pi) as float
// ---------------------------------------------------------------------------
// A CTA stages kMomTile consecutive points (weight and normal, 16 bytes
// each) in shared memory with coalesced loads, then one thread per leaf sums
// its points in Morton order in FP64.  a * n of two floats is exact in
// double, so fma(a, n, m) rounds exactly like m + a * n.
constexpr int kMomThreads = 128;
constexpr int kMomTile = 2048;  // points per CTA (a multiple of every leaf size)

__device__ __forceinline__ void leaf_moments_body(const float4 *__restrict__ p4,
                                                  const float4 *__restrict__ nrm, int64_t n,
                                                  int64_t nleaf, int bucket, double *M,
                                                  int64_t bid)
{
    __shared__ float4 an[kMomTile];  // (nx, ny, nz, a)
    const int64_t p0 = bid * kMomTile;
    for (int t = threadIdx.x; t < kMomTile; t += kMomThreads) {
        const int64_t j = p0 + t;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (j < n) {
            v = nrm[j];
            v.w = p4[j].w;
        }
        an[t] = v;
    }
    __syncthreads();
    const int per = kMomTile / bucket;  // leaves of this tile
    if (threadIdx.x >= per) return;
    const int64_t b = bid * per + threadIdx.x;
    if (b >= nleaf) return;
    const int64_t j0 = b * bucket, j1 = min(j0 + bucket, n);
    double mx = 0.0, my = 0.0, mz = 0.0;
    for (int64_t j = j0; j < j1; ++j) {
        const float4 v = an[j - p0];
        const double a = (double)v.w;
        mx = fma(a, (double)v.x, mx);
        my = fma(a, (double)v.y, my);
        mz = fma(a, (double)v.z, mz);
    }
    const int64_t node = nleaf + b;
    M[3 * node] = mx;
    M[3 * node + 1] = my;
    M[3 * node + 2] = mz;
}

__global__ void __launch_bounds__(kMomThreads)
    k_tree_leaf_moments(const float4 *__restrict__ p4, const float4 *__restrict__ nrm, int64_t n,
                        int64_t nleaf, int bucket, double *M)
{
    leaf_moments_body(p4, nrm, n, nleaf, bucket, M, blockIdx.x);
}

__device__ __forceinline__ void level_moments_body(int64_t first, double *M, int64_t bid)
{
    int64_t node = first + bid * blockDim.x + threadIdx.x;
    if (node >= 2 * first) return;
    int64_t l = 2 * node, r = l + 1;
    for (int k = 0; k < 3; ++k) M[3 * node + k] = __dadd_rn(M[3 * l + k], M[3 * r + k]);
}

__global__ void k_tree_level_moments(int64_t first, double *M)
{
    level_moments_body(first, M, blockIdx.x);
}

// m = M / (4 pi) as float; frec (may be NULL): the node as a 48-byte source
// record (c and m, each value twice) like the point records, for the list
// evaluation's bulk copies
__device__ __forceinline__ void moment_records_body(int64_t nn, const double *M, const float4 *rec,
                                                    float4 *mrec, float4 *frec, int64_t bid)
{
    int64_t node = bid * blockDim.x + threadIdx.x;
    if (node >= nn) return;
    const double fpi = 4.0 * kPi;
    const float mx = (float)__ddiv_rn(M[3 * node], fpi), my = (float)__ddiv_rn(M[3 * node + 1], fpi),
                mz = (float)__ddiv_rn(M[3 * node + 2], fpi);
    mrec[node] = make_float4(mx, my, mz, 0.f);
    if (frec) {
        const float4 c = rec[node];
        frec[3 * node + 0] = make_float4(c.x, c.x, c.y, c.y);
        frec[3 * node + 1] = make_float4(c.z, c.z, mx, mx);
        frec[3 * node + 2] = make_float4(my, my, mz, mz);
    }
}

__global__ void k_tree_moment_records(int64_t nn, const double *M, const float4 *rec, float4 *mrec,
                                      float4 *frec)
{
    moment_records_body(nn, M, rec, mrec, frec, blockIdx.x);
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

// One term; with CLAMP the modified kernel of Sec. 5.2 (eps2 is 0 then):
// rho^2 = max(|p - q|^2, d2), and inside the radius the gradient keeps only
// its -F m / rho^3 part.  Far nodes pass d2 = 0.
template <bool GRAD, bool SCREENED, bool CLAMP = false>
__device__ __forceinline__ void tree_term(TreeAcc &A, float qx, float qy, float qz, float px,
                                          float py, float pz, float mx, float my, float mz,
                                          const EvalParams &ep, float d2 = 0.f)
{
    float dx = px - qx, dy = py - qy, dz = pz - qz;
    float rr = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, ep.eps2)));
    const bool outside = !CLAMP || rr >= d2;
    if (CLAMP) rr = fmaxf(rr, d2);
    float inv = rsqrt_approx(rr);
    float md = fmaf(mz, dz, fmaf(my, dy, mx * dx));
    float i2 = inv * inv;
    if (!SCREENED) {
        float i3 = i2 * inv;
        float phi = md * i3;
        A.tw += phi;
        if (GRAD) {
            float c = outside ? phi * i2 : 0.f;
            A.t1x = fmaf(c, dx, A.t1x); A.t1y = fmaf(c, dy, A.t1y); A.t1z = fmaf(c, dz, A.t1z);
            A.t2x = fmaf(mx, i3, A.t2x); A.t2y = fmaf(my, i3, A.t2y); A.t2z = fmaf(mz, i3, A.t2z);
        }
    } else {
        // g = F / rho^3 = e inv^2 (inv + s), as the packed evaluators
        float rho = rr * inv;
        float e = ex2_approx(rho * ep.nl2e_s);
        float g = (i2 * (inv + ep.s)) * e;
        A.tw = fmaf(g, md, A.tw);
        if (GRAD) {
            float cc = fmaf(3.f, g, e * (ep.s2 * inv));
            float c = outside ? md * (i2 * cc) : 0.f;
            A.t1x = fmaf(c, dx, A.t1x); A.t1y = fmaf(c, dy, A.t1y); A.t1z = fmaf(c, dz, A.t1z);
            A.t2x = fmaf(mx, g, A.t2x); A.t2y = fmaf(my, g, A.t2y); A.t2z = fmaf(mz, g, A.t2z);
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

template <bool GRAD, bool SCREENED, bool CLAMP = false>
__global__ void __launch_bounds__(kTreeThreads)
    k_tree_gwn(const float4 *__restrict__ q, int64_t m, const float4 *__restrict__ rec,
               const float4 *__restrict__ mrec, const float *__restrict__ src, int64_t n,
               int levels, int bucket, EvalParams ep, float *__restrict__ part, int64_t stride,
               unsigned long long *__restrict__ counter, int *err, const IterState *st,
               const float *__restrict__ delta2 = nullptr)
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
            tree_term<GRAD, SCREENED, CLAMP>(A, qq.x, qq.y, qq.z, cr.x, cr.y, cr.z, mm.x, mm.y,
                                             mm.z, ep);
            ++evals;
        }
        const unsigned near = __ballot_sync(0xffffffffu, active && !far);
        if (near) {
            if (node >= nleaf) {
                int64_t j0 = (int64_t)(node - nleaf) * bucket, j1 = min(j0 + bucket, n);
                if (near & lanebit) {
                    for (int64_t j = j0; j < j1; ++j) {
                        const float *r = src + j * kSrcFloats;
                        tree_term<GRAD, SCREENED, CLAMP>(A, qq.x, qq.y, qq.z, r[0], r[2], r[4],
                                                         r[6], r[8], r[10], ep,
                                                         CLAMP ? __ldg(&delta2[j]) : 0.f);
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
// group traversal
// ---------------------------------------------------------------------------
constexpr int kGrpWarps = 4;        // warps per CTA (independent groups)
constexpr int kGrpQ = 64;           // queries per warp group (two per lane)
constexpr int kGrpStack = 1024;     // node stack entries per warp
constexpr int kGrpFar = 64;         // far-node records per flush
constexpr int kGrpNear = 128;       // near-point records per flush

struct GrpSmem {
    int stack[kGrpWarps][kGrpStack];
    float4 far[kGrpWarps][kGrpFar * 3];   // duplicated records, as the sources
    float4 near[kGrpWarps][kGrpNear * 3];
};

struct GrpAcc {
    f2 hw, lw, hgx, lgx, hgy, lgy, hgz, lgz;
};

// One query pair's plain FP32 sums over the records of a flush.
struct PairSums {
    f2 tw, t1x, t1y, t1z, t2x, t2y, t2z;
};

__device__ __forceinline__ void pair_zero(PairSums &T)
{
    T.tw = T.t1x = T.t1y = T.t1z = T.t2x = T.t2y = T.t2z = 0ull;  // +0.0f in both lanes
}

// One record (r0 = (x,x)(y,y), r1 = (z,z)(mx,mx), r2v = (my,my)(mz,mz), d2c the
// modified kernel's (d2,d2)) against one query pair.
template <bool GRAD, bool SCREENED, bool CLAMP>
__device__ __forceinline__ void pair_term(PairSums &T, const ulonglong2 &r0, const ulonglong2 &r1,
                                          const ulonglong2 &r2v, f2 d2c, f2 qx, f2 qy, f2 qz,
                                          f2 eps2, f2 three, f2 sv, f2 s2v, f2 nl2e)
{
    f2 dx = sub2(r0.x, qx);
    f2 dy = sub2(r0.y, qy);
    f2 dz = sub2(r1.x, qz);
    f2 rr = fma2(dx, dx, eps2);
    rr = fma2(dy, dy, rr);
    rr = fma2(dz, dz, rr);
    const f2 r2raw = rr;
    if (CLAMP) rr = max2(rr, d2c);
    f2 inv = rsqrt2(rr);
    f2 md = mul2(r1.y, dx);
    md = fma2(r2v.x, dy, md);
    md = fma2(r2v.y, dz, md);
    f2 i2 = mul2(inv, inv);
    if (!SCREENED) {
        f2 i3 = mul2(i2, inv);
        if (GRAD) {
            f2 phi = mul2(md, i3);
            T.tw = add2(T.tw, phi);
            f2 c = mul2(phi, i2);
            if (CLAMP) c = keep_ge(c, r2raw, d2c);
            T.t1x = fma2(c, dx, T.t1x);
            T.t1y = fma2(c, dy, T.t1y);
            T.t1z = fma2(c, dz, T.t1z);
            T.t2x = fma2(r1.y, i3, T.t2x);
            T.t2y = fma2(r2v.x, i3, T.t2y);
            T.t2z = fma2(r2v.y, i3, T.t2z);
        } else {
            T.tw = fma2(md, i3, T.tw);
        }
    } else {
        // g = F / rho^3 = e inv^2 (inv + s); the gradient's coefficient
        // md (3 F / rho^5 + s^2 e / rho^3) = md inv^2 (3 g + s^2 e inv)
        f2 rho = mul2(rr, inv);
        f2 e = ex22(mul2(rho, nl2e));
        f2 g = mul2(mul2(i2, add2(inv, sv)), e);
        T.tw = fma2(g, md, T.tw);
        if (GRAD) {
            f2 cc = fma2(three, g, mul2(e, mul2(s2v, inv)));
            f2 c = mul2(md, mul2(i2, cc));
            if (CLAMP) c = keep_ge(c, r2raw, d2c);
            T.t1x = fma2(c, dx, T.t1x);
            T.t1y = fma2(c, dy, T.t1y);
            T.t1z = fma2(c, dz, T.t1z);
            T.t2x = fma2(r1.y, g, T.t2x);
            T.t2y = fma2(r2v.x, g, T.t2y);
            T.t2z = fma2(r2v.y, g, T.t2z);
        }
    }
}

// a flush's plain sums folded into the compensated totals
template <bool GRAD, bool SCREENED>
__device__ __forceinline__ void pair_fold(GrpAcc &A, const PairSums &T, f2 three)
{
    two_sum_acc(A.hw, A.lw, T.tw);
    if (GRAD) {
        f2 gx, gy, gz;
        if (!SCREENED) {
            gx = sub2(mul2(three, T.t1x), T.t2x);
            gy = sub2(mul2(three, T.t1y), T.t2y);
            gz = sub2(mul2(three, T.t1z), T.t2z);
        } else {
            gx = sub2(T.t1x, T.t2x);
            gy = sub2(T.t1y, T.t2y);
            gz = sub2(T.t1z, T.t2z);
        }
        two_sum_acc(A.hgx, A.lgx, gx);
        two_sum_acc(A.hgy, A.lgy, gy);
        two_sum_acc(A.hgz, A.lgz, gz);
    }
}

// every lane: its two queries against `cnt` records of `buf`, the flush's
// plain FP32 sums folded into the compensated totals
// With CLAMP the records are four 16-byte words, the fourth (d2, d2, 0, 0)
// (d2 = 0 for far nodes), and the terms are those of the modified kernel.
// UNROLL: records in flight per loop trip (8 in the list evaluation, 3 %
// faster than 4 there; 4 in the on-the-fly group walk, which spills at 8).
template <bool GRAD, bool SCREENED, bool CLAMP = false, int UNROLL = 4>
__device__ __forceinline__ void grp_flush(GrpAcc &A, const float4 *buf, int cnt, f2 qx, f2 qy,
                                          f2 qz, const EvalParams &ep)
{
    constexpr int RW = CLAMP ? 4 : 3;
    const f2 eps2 = pk(ep.eps2, ep.eps2);
    const f2 three = pk(3.f, 3.f);
    const f2 sv = pk(ep.s, ep.s);
    const f2 s2v = pk(ep.s2, ep.s2);
    const f2 nl2e = pk(ep.nl2e_s, ep.nl2e_s);
    PairSums T;
    pair_zero(T);
    const ulonglong2 *rec = reinterpret_cast<const ulonglong2 *>(buf);
#pragma unroll UNROLL
    for (int j = 0; j < cnt; ++j) {
        const ulonglong2 r0 = rec[RW * j + 0];
        const ulonglong2 r1 = rec[RW * j + 1];
        const ulonglong2 r2v = rec[RW * j + 2];
        const f2 d2c = CLAMP ? rec[RW * j + 3].x : 0ull;
        pair_term<GRAD, SCREENED, CLAMP>(T, r0, r1, r2v, d2c, qx, qy, qz, eps2, three, sv, s2v,
                                         nl2e);
    }
    pair_fold<GRAD, SCREENED>(A, T, three);
}

// The warp's 64 queries (two per lane, tail queries repeat the last one) and
// their bounding box (exact min / max of the float coordinates).
struct GrpQueries {
    int64_t ia, ib;
    int nvalid;
    float4 qa, qb;
    float lox, loy, loz, hix, hiy, hiz;
};

__device__ __forceinline__ GrpQueries grp_queries(const float4 *__restrict__ q, int64_t m,
                                                  int64_t q0, int lane)
{
    GrpQueries G;
    G.ia = q0 + lane;
    G.ib = q0 + 32 + lane;
    G.qa = q[min(G.ia, m - 1)];
    G.qb = q[min(G.ib, m - 1)];
    G.nvalid = (int)min((int64_t)kGrpQ, m - q0);
    G.lox = fminf(G.qa.x, G.qb.x); G.loy = fminf(G.qa.y, G.qb.y); G.loz = fminf(G.qa.z, G.qb.z);
    G.hix = fmaxf(G.qa.x, G.qb.x); G.hiy = fmaxf(G.qa.y, G.qb.y); G.hiz = fmaxf(G.qa.z, G.qb.z);
    for (int o = 16; o > 0; o >>= 1) {
        G.lox = fminf(G.lox, __shfl_xor_sync(0xffffffffu, G.lox, o));
        G.loy = fminf(G.loy, __shfl_xor_sync(0xffffffffu, G.loy, o));
        G.loz = fminf(G.loz, __shfl_xor_sync(0xffffffffu, G.loz, o));
        G.hix = fmaxf(G.hix, __shfl_xor_sync(0xffffffffu, G.hix, o));
        G.hiy = fmaxf(G.hiy, __shfl_xor_sync(0xffffffffu, G.hiy, o));
        G.hiz = fmaxf(G.hiz, __shfl_xor_sync(0xffffffffu, G.hiz, o));
    }
    return G;
}

// One warp walks the tree for its group, 32 nodes per step (one per lane).
// A node far from the group's box goes to on_far, a near leaf to on_near,
// an open node pushes its children.  on_far(is_far, node, record, mask) is
// called by every lane each step (warp-uniform); on_near(leaf) once per
// near leaf, by every lane.  Returns false if the stack would overflow.
template <class FarFn, class NearFn>
__device__ __forceinline__ bool grp_walk(int *stack, const float4 *__restrict__ rec,
                                         int64_t nleaf, const GrpQueries &G, int lane,
                                         FarFn &&on_far, NearFn &&on_near)
{
    const unsigned lt = (1u << lane) - 1u;
    int sp = 1;
    if (lane == 0) stack[0] = 1;
    __syncwarp();
    while (sp > 0) {
        const int k = min(sp, 32);
        sp -= k;
        const int node = lane < k ? stack[sp + lane] : 0;
        __syncwarp();  // every pop is read before pushes overwrite the slots
        int act = 0;   // 1 far, 2 near leaf, 3 open
        float4 cr = make_float4(0.f, 0.f, 0.f, -1.f);
        if (lane < k) {
            cr = rec[node];
            if (cr.w >= 0.f) {
                float ex = fmaxf(fmaxf(__fsub_rn(G.lox, cr.x), __fsub_rn(cr.x, G.hix)), 0.f);
                float ey = fmaxf(fmaxf(__fsub_rn(G.loy, cr.y), __fsub_rn(cr.y, G.hiy)), 0.f);
                float ez = fmaxf(fmaxf(__fsub_rn(G.loz, cr.z), __fsub_rn(cr.z, G.hiz)), 0.f);
                float d2 = fmaf(ez, ez, fmaf(ey, ey, __fmul_rn(ex, ex)));
                act = d2 > cr.w ? 1 : ((int64_t)node >= nleaf ? 2 : 3);
            }
        }
        on_far(act == 1, node, cr, __ballot_sync(0xffffffffu, act == 1));
        const unsigned om = __ballot_sync(0xffffffffu, act == 3);
        const int no = __popc(om);
        if (sp + 2 * no > kGrpStack) return false;
        if (act == 3) {
            const int pos = sp + 2 * __popc(om & lt);
            stack[pos] = 2 * node + 1;
            stack[pos + 1] = 2 * node;
        }
        sp += 2 * no;
        unsigned nm = __ballot_sync(0xffffffffu, act == 2);
        while (nm) {
            const int leader = __ffs(nm) - 1;
            nm &= nm - 1;
            on_near(__shfl_sync(0xffffffffu, node, leader));
        }
        __syncwarp();
    }
    return true;
}

template <bool GRAD>
__device__ __forceinline__ void grp_write(const GrpAcc &A, const GrpQueries &G, int64_t m,
                                          float *__restrict__ part, int64_t stride)
{
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int64_t i = h ? G.ib : G.ia;
        if (i >= m) continue;
        float a, b;
        upk(A.hw, a, b); part[0 * stride + i] = h ? b : a;
        upk(A.lw, a, b); part[1 * stride + i] = h ? b : a;
        if (GRAD) {
            upk(A.hgx, a, b); part[2 * stride + i] = h ? b : a;
            upk(A.lgx, a, b); part[3 * stride + i] = h ? b : a;
            upk(A.hgy, a, b); part[4 * stride + i] = h ? b : a;
            upk(A.lgy, a, b); part[5 * stride + i] = h ? b : a;
            upk(A.hgz, a, b); part[6 * stride + i] = h ? b : a;
            upk(A.lgz, a, b); part[7 * stride + i] = h ? b : a;
        }
    }
}

// a near leaf's point records appended to a shared buffer (flushing it when
// full); `flush(cnt)` evaluates the buffer
template <class FlushFn>
__device__ __forceinline__ void grp_take_leaf(const float4 *__restrict__ src4, int64_t j0, int cnt,
                                              float4 *nearb, int &near_cnt, int lane,
                                              FlushFn &&flush)
{
    int done = 0;
    while (done < cnt) {
        const int take = min(cnt - done, kGrpNear - near_cnt);
        if (take == 0) {
            __syncwarp();
            flush(near_cnt);
            near_cnt = 0;
            __syncwarp();
            continue;
        }
        const float4 *from = src4 + 3 * (j0 + done);
        float4 *to = nearb + 3 * near_cnt;
        for (int t = lane; t < 3 * take; t += 32) to[t] = from[t];
        near_cnt += take;
        done += take;
    }
}

template <bool GRAD, bool SCREENED>
__global__ void __launch_bounds__(32 * kGrpWarps)
    k_tree_group(const float4 *__restrict__ q, int64_t m, const float4 *__restrict__ rec,
                 const float4 *__restrict__ mrec, const float *__restrict__ src, int64_t n,
                 int levels, int bucket, EvalParams ep, float *__restrict__ part, int64_t stride,
                 unsigned long long *__restrict__ counter, int *err, const IterState *st)
{
    if (st && cloud_idle(st)) return;  // finished cloud of a batch
    extern __shared__ __align__(16) unsigned char grp_smem_raw[];
    GrpSmem &S = *reinterpret_cast<GrpSmem *>(grp_smem_raw);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t q0 = ((int64_t)blockIdx.x * kGrpWarps + wid) * kGrpQ;
    if (q0 >= m) return;  // the whole warp
    const GrpQueries G = grp_queries(q, m, q0, lane);
    const f2 qx = pk(G.qa.x, G.qb.x), qy = pk(G.qa.y, G.qb.y), qz = pk(G.qa.z, G.qb.z);
    const f2 zero = pk(0.f, 0.f);
    GrpAcc A;
    A.hw = A.lw = A.hgx = A.lgx = A.hgy = A.lgy = A.hgz = A.lgz = zero;
    float4 *farb = S.far[wid];
    float4 *nearb = S.near[wid];
    const float4 *src4 = reinterpret_cast<const float4 *>(src);
    const int64_t nleaf = (int64_t)1 << levels;
    const unsigned lt = (1u << lane) - 1u;
    unsigned long long terms = 0;  // terms per query of the group (warp-uniform)
    int far_cnt = 0, near_cnt = 0;
    auto flush_near = [&](int cnt) {
        grp_flush<GRAD, SCREENED>(A, nearb, cnt, qx, qy, qz, ep);
        terms += (unsigned long long)cnt;
    };
    const bool ok = grp_walk(
        S.stack[wid], rec, nleaf, G, lane,
        [&](bool is_far, int node, const float4 &cr, unsigned fm) {
            // far nodes: dipole records (c, M / 4 pi), duplicated for the packed loop
            const int nf = __popc(fm);
            if (far_cnt + nf > kGrpFar) {
                __syncwarp();
                grp_flush<GRAD, SCREENED>(A, farb, far_cnt, qx, qy, qz, ep);
                terms += (unsigned long long)far_cnt;
                far_cnt = 0;
                __syncwarp();
            }
            if (is_far) {
                const float4 mm = mrec[node];
                float4 *r = farb + 3 * (far_cnt + __popc(fm & lt));
                r[0] = make_float4(cr.x, cr.x, cr.y, cr.y);
                r[1] = make_float4(cr.z, cr.z, mm.x, mm.x);
                r[2] = make_float4(mm.y, mm.y, mm.z, mm.z);
            }
            far_cnt += nf;
        },
        [&](int leaf) {
            const int64_t j0 = ((int64_t)leaf - nleaf) * bucket;
            grp_take_leaf(src4, j0, (int)min((int64_t)bucket, n - j0), nearb, near_cnt, lane,
                          flush_near);
        });
    if (!ok) {
        if (lane == 0) atomicOr(err, kErrStack);
        return;
    }
    __syncwarp();
    if (far_cnt) grp_flush<GRAD, SCREENED>(A, farb, far_cnt, qx, qy, qz, ep);
    if (near_cnt) grp_flush<GRAD, SCREENED>(A, nearb, near_cnt, qx, qy, qz, ep);
    terms += (unsigned long long)(far_cnt + near_cnt);
    grp_write<GRAD>(A, G, m, part, stride);
    if (lane == 0 && counter) atomicAdd(counter, terms * (unsigned long long)G.nvalid);
}

// ---------------------------------------------------------------------------
// interaction lists: node centres and radii depend on the positions only, so
// each group's far nodes and near leaves are the same in every iteration.
// They are found once (a counting walk, a scan, a filling walk) and each
// iteration only evaluates them.
// ---------------------------------------------------------------------------
constexpr int kListWarps = 8;

template <bool FILL>
__global__ void __launch_bounds__(32 * kListWarps)
    k_tree_lists(const float4 *__restrict__ q, int64_t m, const float4 *__restrict__ rec,
                 int levels, int64_t *far_n, int64_t *near_n, int *__restrict__ far_ids,
                 int *__restrict__ near_ids, int *err)
{
    __shared__ int stack[kListWarps][kGrpStack];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t g = (int64_t)blockIdx.x * kListWarps + wid;
    const int64_t q0 = g * kGrpQ;
    if (q0 >= m) return;
    const GrpQueries G = grp_queries(q, m, q0, lane);
    const int64_t nleaf = (int64_t)1 << levels;
    const unsigned lt = (1u << lane) - 1u;
    // FILL: far_n / near_n hold each group's first slot; else they get counts
    int64_t nf = FILL ? far_n[g] : 0, nn = FILL ? near_n[g] : 0;
    const bool ok = grp_walk(
        stack[wid], rec, nleaf, G, lane,
        [&](bool is_far, int node, const float4 &, unsigned fm) {
            if (FILL && is_far) far_ids[nf + __popc(fm & lt)] = node;
            nf += __popc(fm);
        },
        [&](int leaf) {
            if (FILL && lane == 0) near_ids[nn] = leaf;
            ++nn;
        });
    if (!ok) {
        if (lane == 0) atomicOr(err, kErrStack);
        return;
    }
    if (!FILL && lane == 0) {
        far_n[g] = nf;
        near_n[g] = nn;
    }
}

// Evaluation of the lists.  A group's terms are one stream of 48-byte
// records: its far nodes (frec) followed by its near leaves' points (the
// source records; every leaf is read whole -- the last, partial leaf runs
// into the padding records, which have zero moment and add exactly 0).  The
// warp copies the stream in chunks of 64 records into shared memory with
// cp.async (each lane two records, six 16-byte copies), double-buffered so
// that the copy of chunk k+1 overlaps the packed evaluation of chunk k.
constexpr int kLstChunk = 64;

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// global address of record r of the group's stream (point records of
// NEAR_W 16-byte words: 3, or 4 with the modified kernel's radius)
template <int NEAR_W = 3>
__device__ __forceinline__ const float4 *lst_record(int64_t r, int64_t nf, int64_t f0, int64_t e0,
                                                    const int *__restrict__ far_ids,
                                                    const int *__restrict__ near_ids,
                                                    const float4 *__restrict__ frec,
                                                    const float4 *__restrict__ src4, int64_t nleaf,
                                                    int lg_bucket)
{
    if (r < nf) return frec + 3 * (int64_t)far_ids[f0 + r];
    const int64_t rr = r - nf;  // leaves hold 2^lg_bucket points
    const int64_t leaf = near_ids[e0 + (rr >> lg_bucket)];
    return src4 + NEAR_W * (((leaf - nleaf) << lg_bucket) + (rr & ((1 << lg_bucket) - 1)));
}

// Work items: a group's stream is cut into items of at most kItemRecords
// records so that no warp is left with a group whose box straddles a jump
// of the Morton order (such a group opens most of the tree and would keep
// one warp busy long after the rest of the grid has finished).  Each item
// writes its (hi, lo) sums for the group's 64 queries; k_tree_combine adds
// the items of a group in order (deterministic).
constexpr int kItemRecords = 2048;

__global__ void k_tree_items(const int64_t *__restrict__ far_off, const int64_t *__restrict__ near_off,
                             int64_t ng, int bucket, int64_t *__restrict__ cnt)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    const int64_t total = (far_off[g + 1] - far_off[g]) + (near_off[g + 1] - near_off[g]) * bucket;
    cnt[g] = max((int64_t)1, (total + kItemRecords - 1) / kItemRecords);
}

__global__ void k_tree_item_table(const int64_t *__restrict__ item_off, int64_t ng,
                                  int2 *__restrict__ items)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    for (int64_t i = item_off[g], j = 0; i < item_off[g + 1]; ++i, ++j)
        items[i] = make_int2((int)g, (int)(j * kItemRecords));
}

template <bool GRAD, bool SCREENED, bool CLAMP = false>
__device__ __forceinline__ void eval_lists_body(
    const float4 *__restrict__ q, int64_t m, const float4 *__restrict__ frec,
    const float *__restrict__ src, int64_t n, int levels, int bucket,
    const int64_t *__restrict__ far_off, const int *__restrict__ far_ids,
    const int64_t *__restrict__ near_off, const int *__restrict__ near_ids,
    const int2 *__restrict__ items, int64_t nitems, const EvalParams &ep,
    float *__restrict__ ipart, unsigned long long *__restrict__ counter, const IterState *st,
    int64_t bid)
{
    if (st && cloud_idle(st)) return;  // finished cloud of a batch
    constexpr int NA = GRAD ? 4 : 1;
    constexpr int RW = CLAMP ? 4 : 3;  // 16-byte words per staged record
    __shared__ float4 buf_all[kGrpWarps][2][kLstChunk * RW];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t it = bid * kGrpWarps + wid;
    if (it >= nitems) return;
    const int2 item = items[it];
    const int64_t g = item.x;
    const int64_t q0 = g * kGrpQ;
    const GrpQueries G = grp_queries(q, m, q0, lane);
    const f2 qx = pk(G.qa.x, G.qb.x), qy = pk(G.qa.y, G.qb.y), qz = pk(G.qa.z, G.qb.z);
    const f2 zero = pk(0.f, 0.f);
    GrpAcc A;
    A.hw = A.lw = A.hgx = A.lgx = A.hgy = A.lgy = A.hgz = A.lgz = zero;
    const float4 *src4 = reinterpret_cast<const float4 *>(src);
    const int64_t nleaf = (int64_t)1 << levels;
    const int64_t f0 = far_off[g], nf = far_off[g + 1] - f0;
    const int64_t e0 = near_off[g], ne = near_off[g + 1] - e0;
    const int lg_bucket = __ffs(bucket) - 1;  // leaf sizes are powers of two
    const int64_t r_begin = item.y;
    const int64_t r_end = min(r_begin + kItemRecords, nf + ne * bucket);
    const int64_t nchunks = (r_end - r_begin + kLstChunk - 1) / kLstChunk;
    auto issue = [&](int64_t chunk) {
        float4 *b = buf_all[wid][chunk & 1];
        const int64_t r0 = r_begin + chunk * kLstChunk;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int t = lane + 32 * h;
            if (r0 + t < r_end) {
                const float4 *from = lst_record<RW>(r0 + t, nf, f0, e0, far_ids, near_ids, frec,
                                                    src4, nleaf, lg_bucket);
                cp_async16(b + RW * t + 0, from + 0);
                cp_async16(b + RW * t + 1, from + 1);
                cp_async16(b + RW * t + 2, from + 2);
                if (CLAMP) {
                    if (r0 + t < nf) b[RW * t + 3] = make_float4(0.f, 0.f, 0.f, 0.f);  // far node
                    else cp_async16(b + RW * t + 3, from + 3);
                }
            }
        }
        cp_async_commit();
    };
    if (nchunks > 0) issue(0);
    for (int64_t k = 0; k < nchunks; ++k) {
        if (k + 1 < nchunks) issue(k + 1);
        else cp_async_commit();  // an empty group keeps the wait count uniform
        cp_async_wait1();        // chunk k has landed (this lane's copies)
        __syncwarp();            // ... and every lane's
        const int cnt = (int)min((int64_t)kLstChunk, r_end - r_begin - k * kLstChunk);
        grp_flush<GRAD, SCREENED, CLAMP, 8>(A, buf_all[wid][k & 1], cnt, qx, qy, qz, ep);
        __syncwarp();  // buffer k & 1 is reused by the copy of chunk k + 2
    }
    // the item's sums: ipart[((it * NA + a) * 2 + h) * 64 + slot]
    float *o = ipart + it * (int64_t)NA * 2 * kGrpQ;
#pragma unroll
    for (int h2 = 0; h2 < 2; ++h2) {
        const int slot = lane + 32 * h2;
        float a, b;
        upk(A.hw, a, b); o[0 * kGrpQ + slot] = h2 ? b : a;
        upk(A.lw, a, b); o[1 * kGrpQ + slot] = h2 ? b : a;
        if (GRAD) {
            upk(A.hgx, a, b); o[2 * kGrpQ + slot] = h2 ? b : a;
            upk(A.lgx, a, b); o[3 * kGrpQ + slot] = h2 ? b : a;
            upk(A.hgy, a, b); o[4 * kGrpQ + slot] = h2 ? b : a;
            upk(A.lgy, a, b); o[5 * kGrpQ + slot] = h2 ? b : a;
            upk(A.hgz, a, b); o[6 * kGrpQ + slot] = h2 ? b : a;
            upk(A.lgz, a, b); o[7 * kGrpQ + slot] = h2 ? b : a;
        }
    }
    if (counter && r_begin == 0) {
        // terms per query of the whole group: far nodes and the leaves' real points
        int64_t pts = 0;
        for (int64_t e = lane; e < ne; e += 32) {
            const int64_t j0 = ((int64_t)near_ids[e0 + e] - nleaf) * bucket;
            pts += min((int64_t)bucket, n - j0);
        }
        for (int o2 = 16; o2 > 0; o2 >>= 1) pts += __shfl_xor_sync(0xffffffffu, pts, o2);
        if (lane == 0)
            atomicAdd(counter, (unsigned long long)(nf + pts) * (unsigned long long)G.nvalid);
    }
}

template <bool GRAD, bool SCREENED, bool CLAMP = false>
__global__ void __launch_bounds__(32 * kGrpWarps)
    k_tree_eval_lists(const float4 *__restrict__ q, int64_t m, const float4 *__restrict__ frec,
                      const float *__restrict__ src, int64_t n, int levels, int bucket,
                      const int64_t *__restrict__ far_off, const int *__restrict__ far_ids,
                      const int64_t *__restrict__ near_off, const int *__restrict__ near_ids,
                      const int2 *__restrict__ items, int64_t nitems, EvalParams ep,
                      float *__restrict__ ipart, unsigned long long *__restrict__ counter,
                      const IterState *st)
{
    eval_lists_body<GRAD, SCREENED, CLAMP>(q, m, frec, src, n, levels, bucket, far_off, far_ids,
                                           near_off, near_ids, items, nitems, ep, ipart, counter,
                                           st, blockIdx.x);
}

// per query: the items of its group added in order (two-sum on the hi
// parts, lo parts summed), written as the chunk-0 partials of the reduce
template <bool GRAD>
__device__ __forceinline__ void combine_body(const float *__restrict__ ipart,
                                             const int64_t *__restrict__ item_off, int64_t m,
                                             float *__restrict__ part, int64_t stride,
                                             const IterState *st, int64_t bid)
{
    if (st && cloud_idle(st)) return;
    constexpr int NA = GRAD ? 4 : 1;
    const int64_t i = bid * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int64_t g = i / kGrpQ, slot = i % kGrpQ;
    float h[NA], l[NA];
    for (int a = 0; a < NA; ++a) { h[a] = 0.f; l[a] = 0.f; }
    for (int64_t it = item_off[g]; it < item_off[g + 1]; ++it) {
        const float *o = ipart + it * (int64_t)NA * 2 * kGrpQ;
        for (int a = 0; a < NA; ++a) {
            two_sum1(h[a], l[a], o[(2 * a) * kGrpQ + slot]);
            l[a] = __fadd_rn(l[a], o[(2 * a + 1) * kGrpQ + slot]);
        }
    }
    for (int a = 0; a < NA; ++a) {
        part[(2 * a) * stride + i] = h[a];
        part[(2 * a + 1) * stride + i] = l[a];
    }
}

template <bool GRAD>
__global__ void k_tree_combine(const float *__restrict__ ipart, const int64_t *__restrict__ item_off,
                               int64_t m, float *__restrict__ part, int64_t stride,
                               const IterState *st)
{
    combine_body<GRAD>(ipart, item_off, m, part, stride, st, blockIdx.x);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// the group kernels' shared memory (52 KB) is above the default 48 KB limit;
// raised once per device, outside any stream capture (from build_tree)
static cudaError_t group_smem_attr(int dev)
{
    static int done[64] = {0};
    if (dev < 0 || dev >= 64) dev = 0;
    if (done[dev]) return cudaSuccess;
    const int bytes = (int)sizeof(GrpSmem);
    const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(k_tree_group<false, false>, a, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tree_group<false, true>, a, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tree_group<true, false>, a, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tree_group<true, true>, a, bytes);
    if (e == cudaSuccess) done[dev] = 1;
    return e;
}

void free_lists(TreeLists &L)
{
    cudaFree(L.d_item_off);
    cudaFree(L.d_items);
    cudaFree(L.d_ipart);
    cudaFree(L.d_far_off);
    cudaFree(L.d_near_off);
    cudaFree(L.d_far);
    cudaFree(L.d_near);
    L = TreeLists();
}

static uint64_t lists_key(const Ctx *c)
{
    uint32_t bb;
    memcpy(&bb, &c->tree_beta, sizeof bb);
    const uint64_t dg = c->reg_mode == DWG_REG_CLAMP ? (uint64_t)c->delta_gen + 1 : 0;
    return (c->tree_gen * 0x9E3779B97F4A7C15ull) ^ ((uint64_t)bb << 8) ^
           (uint64_t)c->built_depth ^ (dg * 0xC2B2AE3D27D4EB4Full);
}

int tree_lists(Ctx *c, TreeLists &L, const float4 *q, int64_t m, bool *built)
{
    *built = false;
    const uint64_t key = lists_key(c);
    if (L.valid && L.q == q && L.m == m && L.key == key) {
        *built = true;
        return DWG_OK;
    }
    free_lists(L);
    ++c->bufgen;  // a captured graph may hold the old lists
    if (m < 1) return DWG_OK;
    const int64_t ng = ceil_div(m, kGrpQ);
    const unsigned blocks = (unsigned)ceil_div(ng, kListWarps);
    int64_t *cnt_f = nullptr, *cnt_n = nullptr;
    auto run = [&]() -> int {
        DWG_CUDA_TRY(c, cudaMalloc(&cnt_f, ng * sizeof(int64_t)));
        DWG_CUDA_TRY(c, cudaMalloc(&cnt_n, ng * sizeof(int64_t)));
        DWG_CUDA_TRY(c, cudaMalloc(&L.d_far_off, (ng + 1) * sizeof(int64_t)));
        DWG_CUDA_TRY(c, cudaMalloc(&L.d_near_off, (ng + 1) * sizeof(int64_t)));
        k_tree_lists<false><<<blocks, 32 * kListWarps, 0, c->stream>>>(
            q, m, c->d_tree_rec, c->tree_levels, cnt_f, cnt_n, nullptr, nullptr, c->d_err);
        DWG_CUDA_TRY(c, cudaGetLastError());
        int rc = scan_i64(c, cnt_f, L.d_far_off, ng, L.d_far_off + ng);
        if (!rc) rc = scan_i64(c, cnt_n, L.d_near_off, ng, L.d_near_off + ng);
        if (rc) return rc;
        DWG_CUDA_TRY(c, cudaStreamSynchronize(c->stream));  // cnt_f is reused below
        int herr = 0;
        DWG_CUDA_TRY(c, cudaMemcpyAsync(&L.nfar, L.d_far_off + ng, sizeof(int64_t),
                                        cudaMemcpyDeviceToHost, c->stream));
        DWG_CUDA_TRY(c, cudaMemcpyAsync(&L.nnear, L.d_near_off + ng, sizeof(int64_t),
                                        cudaMemcpyDeviceToHost, c->stream));
        DWG_CUDA_TRY(c, cudaMemcpyAsync(&herr, c->d_err, sizeof(int), cudaMemcpyDeviceToHost,
                                        c->stream));
        DWG_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        if (herr) {
            c->err = "tree lists: traversal stack overflow";
            return DWG_ERR_CUDA;
        }
        // the lists stay resident across iterations; take at most half of
        // the free memory, else keep walking the tree every iteration
        size_t free_b = 0, total_b = 0;
        DWG_CUDA_TRY(c, cudaMemGetInfo(&free_b, &total_b));
        const double need = 4.0 * (double)(L.nfar + L.nnear) +
                            (8.0 + 4.0 * 8 * kGrpQ) * ((double)(L.nfar + L.nnear * c->tree_leaf) /
                                                           kItemRecords + (double)ng);
        if (need > 0.5 * (double)free_b) return DWG_OK;
        DWG_CUDA_TRY(c, cudaMalloc(&L.d_far, std::max<int64_t>(L.nfar, 1) * sizeof(int)));
        DWG_CUDA_TRY(c, cudaMalloc(&L.d_near, std::max<int64_t>(L.nnear, 1) * sizeof(int)));
        k_tree_lists<true><<<blocks, 32 * kListWarps, 0, c->stream>>>(
            q, m, c->d_tree_rec, c->tree_levels, L.d_far_off, L.d_near_off, L.d_far, L.d_near,
            c->d_err);
        DWG_CUDA_TRY(c, cudaGetLastError());
        // work items and their partial-sum buffer
        DWG_CUDA_TRY(c, cudaMalloc(&L.d_item_off, (ng + 1) * sizeof(int64_t)));
        k_tree_items<<<(unsigned)ceil_div(ng, 256), 256, 0, c->stream>>>(
            L.d_far_off, L.d_near_off, ng, c->tree_leaf, cnt_f);
        DWG_CUDA_TRY(c, cudaGetLastError());
        if ((rc = scan_i64(c, cnt_f, L.d_item_off, ng, L.d_item_off + ng))) return rc;
        DWG_CUDA_TRY(c, cudaMemcpyAsync(&L.nitems, L.d_item_off + ng, sizeof(int64_t),
                                        cudaMemcpyDeviceToHost, c->stream));
        DWG_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        DWG_CUDA_TRY(c, cudaMalloc(&L.d_items, L.nitems * sizeof(int2)));
        DWG_CUDA_TRY(c, cudaMalloc(&L.d_ipart, L.nitems * 8 * kGrpQ * sizeof(float)));
        k_tree_item_table<<<(unsigned)ceil_div(ng, 256), 256, 0, c->stream>>>(L.d_item_off, ng,
                                                                              L.d_items);
        DWG_CUDA_TRY(c, cudaGetLastError());
        L.q = q;
        L.m = m;
        L.key = key;
        L.valid = true;
        *built = true;
        return DWG_OK;
    };
    int rc = run();
    cudaFree(cnt_f);
    cudaFree(cnt_n);
    if (rc || !L.valid) {
        free_lists(L);
        if (!rc) *built = false;
    }
    return rc;
}

void free_tree(Ctx *c)
{
    free_lists(c->lists_p);
    free_lists(c->lists_c);
    cudaFree(c->d_tree_A);
    cudaFree(c->d_tree_C);
    cudaFree(c->d_tree_R);
    cudaFree(c->d_tree_M);
    cudaFree(c->d_tree_rec);
    cudaFree(c->d_tree_mrec);
    cudaFree(c->d_tree_frec);
    cudaFree(c->d_tree_dmax);
    c->d_tree_frec = nullptr;
    c->d_tree_dmax = nullptr;
    c->d_tree_A = c->d_tree_C = c->d_tree_R = c->d_tree_M = nullptr;
    c->d_tree_rec = c->d_tree_mrec = nullptr;
    c->tree_built = false;
    c->tree_beta_set = -1.0;
}

int build_tree(Ctx *c)
{
    if (c->tree_built) return DWG_OK;
    // leaves of tree_leaf Morton-consecutive points, 2^tree_levels of them
    int64_t nb = ceil_div(c->n, c->tree_leaf);
    int L = 0;
    while (((int64_t)1 << L) < nb) ++L;
    c->tree_levels = L;
    const int64_t nleaf = (int64_t)1 << L, nn = 2 * nleaf;
    const int B = 256;
    free_tree(c);
    DWG_CUDA_TRY(c, group_smem_attr(c->device));
    DWG_CUDA_TRY(c, cudaMalloc(&c->d_tree_A, nn * sizeof(double)));
    DWG_CUDA_TRY(c, cudaMalloc(&c->d_tree_C, 3 * nn * sizeof(double)));
    DWG_CUDA_TRY(c, cudaMalloc(&c->d_tree_R, nn * sizeof(double)));
    DWG_CUDA_TRY(c, cudaMalloc(&c->d_tree_M, 3 * nn * sizeof(double)));
    DWG_CUDA_TRY(c, cudaMalloc(&c->d_tree_rec, nn * sizeof(float4)));
    DWG_CUDA_TRY(c, cudaMalloc(&c->d_tree_mrec, nn * sizeof(float4)));
    DWG_CUDA_TRY(c, cudaMalloc(&c->d_tree_frec, 3 * nn * sizeof(float4)));
    DWG_CUDA_TRY(c, cudaMemsetAsync(c->d_tree_A, 0, nn * sizeof(double), c->stream));
    DWG_CUDA_TRY(c, cudaMemsetAsync(c->d_tree_M, 0, 3 * nn * sizeof(double), c->stream));
    double *Sp = nullptr;
    DWG_CUDA_TRY(c, cudaMalloc(&Sp, 3 * nn * sizeof(double)));
    k_tree_leaf_sums<<<(unsigned)ceil_div(nleaf, B), B, 0, c->stream>>>(
        c->d_p4, c->n, nleaf, c->tree_leaf, c->d_tree_A, Sp);
    for (int lv = L - 1; lv >= 0; --lv) {
        int64_t first = (int64_t)1 << lv;
        k_tree_level_sums<<<(unsigned)ceil_div(first, B), B, 0, c->stream>>>(first, c->d_tree_A, Sp);
    }
    k_tree_centres<<<(unsigned)ceil_div(nn, B), B, 0, c->stream>>>(nn, c->d_tree_A, Sp, c->d_tree_C);
    k_tree_leaf_radius<<<(unsigned)ceil_div(nleaf, B), B, 0, c->stream>>>(
        c->d_p4, c->n, nleaf, c->tree_leaf, c->d_tree_C, c->d_tree_R);
    for (int lv = L - 1; lv >= 0; --lv) {
        int64_t first = (int64_t)1 << lv;
        k_tree_level_radius<<<(unsigned)ceil_div(first, B), B, 0, c->stream>>>(
            first, c->d_tree_A, c->d_tree_C, c->d_tree_R);
    }
    DWG_CUDA_TRY(c, cudaGetLastError());
    DWG_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    cudaFree(Sp);
    c->tree_built = true;
    c->tree_beta_set = -1.0;
    ++c->tree_gen;
    ++c->bufgen;  // a captured graph holds the old node arrays
    return DWG_OK;
}

int tree_records(Ctx *c)
{
    const bool clamp = c->reg_mode == DWG_REG_CLAMP;
    const int dgen = clamp ? c->delta_gen : -1;
    if (c->tree_beta_set == (double)c->tree_beta && c->tree_rec_dgen == dgen) return DWG_OK;
    const int64_t nleaf = (int64_t)1 << c->tree_levels, nn = 2 * nleaf;
    if (clamp) {
        if (!c->d_tree_dmax) DWG_CUDA_TRY(c, cudaMalloc(&c->d_tree_dmax, nn * sizeof(double)));
        k_tree_leaf_dmax<<<(unsigned)ceil_div(nleaf, 256), 256, 0, c->stream>>>(
            c->d_delta2, c->n, nleaf, c->tree_leaf, c->d_tree_dmax);
        for (int64_t first = nleaf / 2; first >= 1; first /= 2)
            k_tree_level_dmax<<<(unsigned)ceil_div(first, 256), 256, 0, c->stream>>>(
                first, c->d_tree_dmax);
    }
    k_tree_records<<<(unsigned)ceil_div(nn, 256), 256, 0, c->stream>>>(
        nn, c->d_tree_A, c->d_tree_C, c->d_tree_R, (double)c->tree_beta,
        clamp ? c->d_tree_dmax : nullptr, c->d_tree_rec);
    DWG_CUDA_TRY(c, cudaGetLastError());
    c->tree_beta_set = (double)c->tree_beta;
    c->tree_rec_dgen = dgen;
    return DWG_OK;
}

cudaError_t launch_tree_moments(Ctx *c)
{
    const int64_t nleaf = (int64_t)1 << c->tree_levels, nn = 2 * nleaf;
    const int B = 256;
    k_tree_leaf_moments<<<(unsigned)ceil_div(nleaf * c->tree_leaf, kMomTile), kMomThreads, 0,
                          c->stream>>>(c->d_p4, c->d_nrm, c->n, nleaf, c->tree_leaf,
                                       c->d_tree_M);
    for (int lv = c->tree_levels - 1; lv >= 0; --lv) {
        int64_t first = (int64_t)1 << lv;
        k_tree_level_moments<<<(unsigned)ceil_div(first, B), B, 0, c->stream>>>(first, c->d_tree_M);
    }
    k_tree_moment_records<<<(unsigned)ceil_div(nn, B), B, 0, c->stream>>>(
        nn, c->d_tree_M, c->d_tree_rec, c->d_tree_mrec, c->d_tree_frec);
    return cudaGetLastError();
}

template <bool GRAD, bool SCREENED>
static cudaError_t launch_group_t(Ctx *c, const float4 *q, int64_t m, float *part, int64_t stride,
                                  const IterState *st)
{
    cudaError_t e = group_smem_attr(c->device);
    if (e != cudaSuccess) return e;
    EvalParams ep = make_eval_params(c);
    const int64_t per_cta = (int64_t)kGrpWarps * kGrpQ;
    k_tree_group<GRAD, SCREENED><<<(unsigned)ceil_div(m, per_cta), 32 * kGrpWarps,
                                    sizeof(GrpSmem), c->stream>>>(
        q, m, c->d_tree_rec, c->d_tree_mrec, c->d_src, c->n, c->tree_levels, c->tree_leaf, ep,
        part, stride, c->d_counter, c->d_err, st);
    return cudaGetLastError();
}

template <bool GRAD, bool SCREENED, bool CLAMP = false>
static cudaError_t launch_lists_t(Ctx *c, const TreeLists &L, float *part, int64_t stride,
                                  const IterState *st)
{
    EvalParams ep = make_eval_params(c);
    k_tree_eval_lists<GRAD, SCREENED, CLAMP><<<(unsigned)ceil_div(L.nitems, kGrpWarps),
                                                32 * kGrpWarps, 0, c->stream>>>(
        L.q, L.m, c->d_tree_frec, CLAMP ? c->d_src16 : c->d_src, c->n, c->tree_levels,
        c->tree_leaf, L.d_far_off, L.d_far, L.d_near_off, L.d_near, L.d_items, L.nitems, ep,
        L.d_ipart, c->d_counter, st);
    k_tree_combine<GRAD><<<(unsigned)ceil_div(L.m, 256), 256, 0, c->stream>>>(
        L.d_ipart, L.d_item_off, L.m, part, stride, st);
    return cudaGetLastError();
}

cudaError_t launch_tree_iter(Ctx *c, TreeLists &L, const float4 *q, int64_t m, bool grad,
                             float *part, int64_t stride, const IterState *st)
{
    if (!(c->tree_group && L.valid && L.q == q && L.m == m && L.key == lists_key(c)))
        return launch_tree_gwn(c, q, m, grad, part, stride, st);
    const bool scr = make_eval_params(c).screened != 0;
    if (c->reg_mode == DWG_REG_CLAMP) {
        if (grad)
            return scr ? launch_lists_t<true, true, true>(c, L, part, stride, st)
                       : launch_lists_t<true, false, true>(c, L, part, stride, st);
        return scr ? launch_lists_t<false, true, true>(c, L, part, stride, st)
                   : launch_lists_t<false, false, true>(c, L, part, stride, st);
    }
    if (grad)
        return scr ? launch_lists_t<true, true>(c, L, part, stride, st)
                   : launch_lists_t<true, false>(c, L, part, stride, st);
    return scr ? launch_lists_t<false, true>(c, L, part, stride, st)
               : launch_lists_t<false, false>(c, L, part, stride, st);
}

// the per-query walk with the modified kernel (also its path when the
// group lists are not available: the on-the-fly group walk has no clamp)
template <bool GRAD, bool SCREENED>
static cudaError_t launch_walk_clamp(Ctx *c, const float4 *q, int64_t m, float *part,
                                     int64_t stride, const IterState *st)
{
    EvalParams ep = make_eval_params(c);
    k_tree_gwn<GRAD, SCREENED, true><<<(unsigned)ceil_div(m, kTreeThreads), kTreeThreads, 0,
                                       c->stream>>>(
        q, m, c->d_tree_rec, c->d_tree_mrec, c->d_src, c->n, c->tree_levels, c->tree_leaf, ep,
        part, stride, c->d_counter, c->d_err, st, c->d_delta2);
    return cudaGetLastError();
}

cudaError_t launch_tree_gwn(Ctx *c, const float4 *q, int64_t m, bool grad, float *part,
                            int64_t stride, const IterState *st)
{
    EvalParams ep = make_eval_params(c);
    if (c->reg_mode == DWG_REG_CLAMP) {
        if (grad)
            return ep.screened ? launch_walk_clamp<true, true>(c, q, m, part, stride, st)
                               : launch_walk_clamp<true, false>(c, q, m, part, stride, st);
        return ep.screened ? launch_walk_clamp<false, true>(c, q, m, part, stride, st)
                           : launch_walk_clamp<false, false>(c, q, m, part, stride, st);
    }
    if (c->tree_group) {
        if (grad)
            return ep.screened ? launch_group_t<true, true>(c, q, m, part, stride, st)
                               : launch_group_t<true, false>(c, q, m, part, stride, st);
        return ep.screened ? launch_group_t<false, true>(c, q, m, part, stride, st)
                           : launch_group_t<false, false>(c, q, m, part, stride, st);
    }
    unsigned blocks = (unsigned)ceil_div(m, kTreeThreads);
    if (grad) {
        if (ep.screened)
            k_tree_gwn<true, true><<<blocks, kTreeThreads, 0, c->stream>>>(
                q, m, c->d_tree_rec, c->d_tree_mrec, c->d_src, c->n, c->tree_levels, c->tree_leaf, ep, part, stride,
                c->d_counter, c->d_err, st);
        else
            k_tree_gwn<true, false><<<blocks, kTreeThreads, 0, c->stream>>>(
                q, m, c->d_tree_rec, c->d_tree_mrec, c->d_src, c->n, c->tree_levels, c->tree_leaf, ep, part, stride,
                c->d_counter, c->d_err, st);
    } else {
        if (ep.screened)
            k_tree_gwn<false, true><<<blocks, kTreeThreads, 0, c->stream>>>(
                q, m, c->d_tree_rec, c->d_tree_mrec, c->d_src, c->n, c->tree_levels, c->tree_leaf, ep, part, stride,
                c->d_counter, c->d_err, st);
        else
            k_tree_gwn<false, false><<<blocks, kTreeThreads, 0, c->stream>>>(
                q, m, c->d_tree_rec, c->d_tree_mrec, c->d_src, c->n, c->tree_levels, c->tree_leaf, ep, part, stride,
                c->d_counter, c->d_err, st);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// batched phases: every tree cloud of a batch in one launch (each cloud's
// blocks as in its own launch)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kMomThreads)
    k_tree_leaf_moments_b(const CloudIter *__restrict__ cl, const int *__restrict__ off, int ncl)
{
    const int ci = seg_cloud(off, ncl);
    const CloudIter &c = cl[ci];
    leaf_moments_body(c.p4, c.nrm_c, c.n, (int64_t)1 << c.levels, c.bucket, c.tree_M,
                      (int64_t)blockIdx.x - off[ci]);
}

__global__ void k_tree_level_moments_b(const CloudIter *__restrict__ cl, const int *__restrict__ off,
                                       int ncl, int level)
{
    const int ci = seg_cloud(off, ncl);
    level_moments_body((int64_t)1 << level, cl[ci].tree_M, (int64_t)blockIdx.x - off[ci]);
}

__global__ void k_tree_moment_records_b(const CloudIter *__restrict__ cl, const int *__restrict__ off,
                                        int ncl)
{
    const int ci = seg_cloud(off, ncl);
    const CloudIter &c = cl[ci];
    moment_records_body((int64_t)2 << c.levels, c.tree_M, c.tree_rec, c.tree_mrec, c.tree_frec,
                        (int64_t)blockIdx.x - off[ci]);
}

// GRAD: the points (w and grad w), else the corners (w).  Held to the
// registers of the single-cloud kernel (8 or 5 resident CTAs per SM): the
// per-cloud arguments come from memory here, not from the parameter bank,
// and would otherwise take registers for the whole item.
template <bool GRAD, bool SCREENED>
__global__ void __launch_bounds__(32 * kGrpWarps, GRAD ? 5 : 8)
    k_tree_eval_lists_b(const CloudIter *__restrict__ cl, const int *__restrict__ off, int ncl)
{
    const int ci = seg_cloud(off, ncl);
    const CloudIter &c = cl[ci];
    constexpr int w = GRAD ? 0 : 1;
    eval_lists_body<GRAD, SCREENED>(c.lq[w], c.lm[w], c.tree_frec, c.src, c.n, c.levels, c.bucket,
                                    c.far_off[w], c.far_ids[w], c.near_off[w], c.near_ids[w],
                                    c.items[w], c.nitems[w], c.ep, c.ipart[w], c.counter, c.st,
                                    (int64_t)blockIdx.x - off[ci]);
}

template <bool GRAD>
__global__ void k_tree_combine_b(const CloudIter *__restrict__ cl, const int *__restrict__ off,
                                 int ncl)
{
    const int ci = seg_cloud(off, ncl);
    const CloudIter &c = cl[ci];
    constexpr int w = GRAD ? 0 : 1;
    combine_body<GRAD>(c.ipart[w], c.item_off[w], c.lm[w], c.lpart[w], c.lm[w], c.st,
                       (int64_t)blockIdx.x - off[ci]);
}

cudaError_t launch_tree_batch(int phase, const CloudIter *cl, const int *off, int ncl,
                              int blocks, int level, bool screened, cudaStream_t s)
{
    if (blocks <= 0) return cudaSuccess;
    const unsigned g = (unsigned)blocks;
    const unsigned T = 32 * kGrpWarps;
    if (level >= 0) {
        k_tree_level_moments_b<<<g, 256, 0, s>>>(cl, off, ncl, level);
        return cudaGetLastError();
    }
    switch (phase) {
    case kPhLeafMom: k_tree_leaf_moments_b<<<g, kMomThreads, 0, s>>>(cl, off, ncl); break;
    case kPhMomRec: k_tree_moment_records_b<<<g, 256, 0, s>>>(cl, off, ncl); break;
    case kPhListsP:
        if (screened) k_tree_eval_lists_b<true, true><<<g, T, 0, s>>>(cl, off, ncl);
        else k_tree_eval_lists_b<true, false><<<g, T, 0, s>>>(cl, off, ncl);
        break;
    case kPhListsC:
        if (screened) k_tree_eval_lists_b<false, true><<<g, T, 0, s>>>(cl, off, ncl);
        else k_tree_eval_lists_b<false, false><<<g, T, 0, s>>>(cl, off, ncl);
        break;
    case kPhCombineP: k_tree_combine_b<true><<<g, 256, 0, s>>>(cl, off, ncl); break;
    case kPhCombineC: k_tree_combine_b<false><<<g, 256, 0, s>>>(cl, off, ncl); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// the group lists of the points (corners = false) or the corners hold for
// the current tree, opening angle and depth (launch_tree_iter's test)
bool tree_lists_current(const Ctx *c, bool corners)
{
    const TreeLists &L = corners ? c->lists_c : c->lists_p;
    const float4 *q = corners ? c->d_corner_pos : c->d_p4;
    const int64_t m = corners ? c->ncorners : c->n;
    return c->tree_group && L.valid && L.q == q && L.m == m && L.key == lists_key(c);
}

// blocks of a cloud's part in a batched tree phase (0: no part); level >= 0:
// the moments of that tree level
int tree_phase_blocks(const Ctx *c, int phase, int level)
{
    if (!use_tree(c) || !c->tree_built) return 0;
    const int64_t nleaf = (int64_t)1 << c->tree_levels, nn = 2 * nleaf;
    if (level >= 0) return level < c->tree_levels ? (int)ceil_div((int64_t)1 << level, 256) : 0;
    const bool lists_p = tree_lists_current(c, false);
    const bool lists_c = c->mode == DWG_UPDATE_LEVELSET && tree_lists_current(c, true);
    switch (phase) {
    case kPhLeafMom: return (int)ceil_div(nleaf * c->tree_leaf, kMomTile);
    case kPhMomRec: return (int)ceil_div(nn, 256);
    case kPhListsP: return lists_p ? (int)ceil_div(c->lists_p.nitems, kGrpWarps) : 0;
    case kPhListsC: return lists_c ? (int)ceil_div(c->lists_c.nitems, kGrpWarps) : 0;
    case kPhCombineP: return lists_p ? (int)ceil_div(c->lists_p.m, 256) : 0;
    case kPhCombineC: return lists_c ? (int)ceil_div(c->lists_c.m, 256) : 0;
    default: return 0;
    }
}

}  // namespace dwg
