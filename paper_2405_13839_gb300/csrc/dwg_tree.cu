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
                                    int64_t n, int64_t nleaf, int bucket, double *M)
{
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nleaf) return;
    int64_t node = nleaf + b, j0 = b * bucket, j1 = min(j0 + bucket, n);
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
               int levels, int bucket, EvalParams ep, float *__restrict__ part, int64_t stride,
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
                int64_t j0 = (int64_t)(node - nleaf) * bucket, j1 = min(j0 + bucket, n);
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

// every lane: its two queries against `cnt` records of `buf`, the flush's
// plain FP32 sums folded into the compensated totals
template <bool GRAD, bool SCREENED>
__device__ __forceinline__ void grp_flush(GrpAcc &A, const float4 *buf, int cnt, f2 qx, f2 qy,
                                          f2 qz, const EvalParams &ep)
{
    const f2 eps2 = pk(ep.eps2, ep.eps2);
    const f2 three = pk(3.f, 3.f);
    const f2 zero = pk(0.f, 0.f);
    const f2 sv = pk(ep.s, ep.s);
    const f2 s2v = pk(ep.s2, ep.s2);
    const f2 nl2e = pk(ep.nl2e_s, ep.nl2e_s);
    f2 tw = zero, t1x = zero, t1y = zero, t1z = zero, t2x = zero, t2y = zero, t2z = zero;
    const ulonglong2 *rec = reinterpret_cast<const ulonglong2 *>(buf);
#pragma unroll 4
    for (int j = 0; j < cnt; ++j) {
        const ulonglong2 r0 = rec[3 * j + 0];  // (x,x) (y,y)
        const ulonglong2 r1 = rec[3 * j + 1];  // (z,z) (mx,mx)
        const ulonglong2 r2v = rec[3 * j + 2]; // (my,my) (mz,mz)
        f2 dx = sub2(r0.x, qx);
        f2 dy = sub2(r0.y, qy);
        f2 dz = sub2(r1.x, qz);
        f2 rr = fma2(dx, dx, eps2);
        rr = fma2(dy, dy, rr);
        rr = fma2(dz, dz, rr);
        f2 inv = rsqrt2(rr);
        f2 md = mul2(r1.y, dx);
        md = fma2(r2v.x, dy, md);
        md = fma2(r2v.y, dz, md);
        f2 i2 = mul2(inv, inv);
        f2 i3 = mul2(i2, inv);
        if (!SCREENED) {
            if (GRAD) {
                f2 phi = mul2(md, i3);
                tw = add2(tw, phi);
                f2 c = mul2(phi, i2);
                t1x = fma2(c, dx, t1x);
                t1y = fma2(c, dy, t1y);
                t1z = fma2(c, dz, t1z);
                t2x = fma2(r1.y, i3, t2x);
                t2y = fma2(r2v.x, i3, t2y);
                t2z = fma2(r2v.y, i3, t2z);
            } else {
                tw = fma2(md, i3, tw);
            }
        } else {
            f2 rho = mul2(rr, inv);
            f2 e = ex22(mul2(rho, nl2e));
            f2 F = fma2(e, mul2(rho, sv), e);
            f2 phi = mul2(md, i3);
            tw = fma2(F, phi, tw);
            if (GRAD) {
                f2 fi3 = mul2(F, i3);
                f2 cc = fma2(three, mul2(F, i2), mul2(s2v, e));
                f2 c = mul2(phi, cc);
                t1x = fma2(c, dx, t1x);
                t1y = fma2(c, dy, t1y);
                t1z = fma2(c, dz, t1z);
                t2x = fma2(r1.y, fi3, t2x);
                t2y = fma2(r2v.x, fi3, t2y);
                t2z = fma2(r2v.y, fi3, t2z);
            }
        }
    }
    two_sum_acc(A.hw, A.lw, tw);
    if (GRAD) {
        f2 gx, gy, gz;
        if (!SCREENED) {
            gx = sub2(mul2(three, t1x), t2x);
            gy = sub2(mul2(three, t1y), t2y);
            gz = sub2(mul2(three, t1z), t2z);
        } else {
            gx = sub2(t1x, t2x);
            gy = sub2(t1y, t2y);
            gz = sub2(t1z, t2z);
        }
        two_sum_acc(A.hgx, A.lgx, gx);
        two_sum_acc(A.hgy, A.lgy, gy);
        two_sum_acc(A.hgz, A.lgz, gz);
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
    const int64_t ia = q0 + lane, ib = q0 + 32 + lane;
    const float4 qa = q[min(ia, m - 1)], qb = q[min(ib, m - 1)];
    const int nvalid = (int)min((int64_t)kGrpQ, m - q0);
    // the group's bounding box (exact min / max of the float coordinates)
    float lox = fminf(qa.x, qb.x), loy = fminf(qa.y, qb.y), loz = fminf(qa.z, qb.z);
    float hix = fmaxf(qa.x, qb.x), hiy = fmaxf(qa.y, qb.y), hiz = fmaxf(qa.z, qb.z);
    for (int o = 16; o > 0; o >>= 1) {
        lox = fminf(lox, __shfl_xor_sync(0xffffffffu, lox, o));
        loy = fminf(loy, __shfl_xor_sync(0xffffffffu, loy, o));
        loz = fminf(loz, __shfl_xor_sync(0xffffffffu, loz, o));
        hix = fmaxf(hix, __shfl_xor_sync(0xffffffffu, hix, o));
        hiy = fmaxf(hiy, __shfl_xor_sync(0xffffffffu, hiy, o));
        hiz = fmaxf(hiz, __shfl_xor_sync(0xffffffffu, hiz, o));
    }
    const f2 qx = pk(qa.x, qb.x), qy = pk(qa.y, qb.y), qz = pk(qa.z, qb.z);
    const f2 zero = pk(0.f, 0.f);
    GrpAcc A;
    A.hw = A.lw = A.hgx = A.lgx = A.hgy = A.lgy = A.hgz = A.lgz = zero;

    int *stack = S.stack[wid];
    float4 *farb = S.far[wid];
    float4 *nearb = S.near[wid];
    const float4 *src4 = reinterpret_cast<const float4 *>(src);
    const int64_t nleaf = (int64_t)1 << levels;
    const unsigned lt = (1u << lane) - 1u;
    unsigned long long terms = 0;  // terms per query of the group (warp-uniform)
    int far_cnt = 0, near_cnt = 0, sp = 1;
    bool overflow = false;
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
                float ex = fmaxf(fmaxf(__fsub_rn(lox, cr.x), __fsub_rn(cr.x, hix)), 0.f);
                float ey = fmaxf(fmaxf(__fsub_rn(loy, cr.y), __fsub_rn(cr.y, hiy)), 0.f);
                float ez = fmaxf(fmaxf(__fsub_rn(loz, cr.z), __fsub_rn(cr.z, hiz)), 0.f);
                float d2 = fmaf(ez, ez, fmaf(ey, ey, __fmul_rn(ex, ex)));
                act = d2 > cr.w ? 1 : ((int64_t)node >= nleaf ? 2 : 3);
            }
        }
        // far nodes: dipole records (c, M / 4 pi), duplicated for the packed loop
        const unsigned fm = __ballot_sync(0xffffffffu, act == 1);
        const int nf = __popc(fm);
        if (far_cnt + nf > kGrpFar) {
            __syncwarp();
            grp_flush<GRAD, SCREENED>(A, farb, far_cnt, qx, qy, qz, ep);
            terms += (unsigned long long)far_cnt;
            far_cnt = 0;
            __syncwarp();
        }
        if (act == 1) {
            const float4 mm = mrec[node];
            float4 *r = farb + 3 * (far_cnt + __popc(fm & lt));
            r[0] = make_float4(cr.x, cr.x, cr.y, cr.y);
            r[1] = make_float4(cr.z, cr.z, mm.x, mm.x);
            r[2] = make_float4(mm.y, mm.y, mm.z, mm.z);
        }
        far_cnt += nf;
        // open nodes: push both children
        const unsigned om = __ballot_sync(0xffffffffu, act == 3);
        const int no = __popc(om);
        if (sp + 2 * no > kGrpStack) {
            overflow = true;
            break;
        }
        if (act == 3) {
            const int pos = sp + 2 * __popc(om & lt);
            stack[pos] = 2 * node + 1;
            stack[pos + 1] = 2 * node;
        }
        sp += 2 * no;
        // near leaves: their points' records, copied in order
        unsigned nm = __ballot_sync(0xffffffffu, act == 2);
        while (nm) {
            const int leader = __ffs(nm) - 1;
            nm &= nm - 1;
            const int leaf = __shfl_sync(0xffffffffu, node, leader);
            const int64_t j0 = ((int64_t)leaf - nleaf) * bucket;
            const int cnt = (int)min((int64_t)bucket, n - j0);
            int done = 0;
            while (done < cnt) {
                const int take = min(cnt - done, kGrpNear - near_cnt);
                if (take == 0) {
                    __syncwarp();
                    grp_flush<GRAD, SCREENED>(A, nearb, near_cnt, qx, qy, qz, ep);
                    terms += (unsigned long long)near_cnt;
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
        __syncwarp();
    }
    if (overflow) {
        if (lane == 0) atomicOr(err, kErrStack);
        return;
    }
    __syncwarp();
    if (far_cnt) grp_flush<GRAD, SCREENED>(A, farb, far_cnt, qx, qy, qz, ep);
    if (near_cnt) grp_flush<GRAD, SCREENED>(A, nearb, near_cnt, qx, qy, qz, ep);
    terms += (unsigned long long)(far_cnt + near_cnt);
    // chunk-0 partials, as the per-query kernel writes them
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int64_t i = h ? ib : ia;
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
    if (lane == 0 && counter) atomicAdd(counter, terms * (unsigned long long)nvalid);
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

void free_tree(Ctx *c)
{
    cudaFree(c->d_tree_A);
    cudaFree(c->d_tree_C);
    cudaFree(c->d_tree_R);
    cudaFree(c->d_tree_M);
    cudaFree(c->d_tree_rec);
    cudaFree(c->d_tree_mrec);
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
    ++c->bufgen;  // a captured graph holds the old node arrays
    return DWG_OK;
}

int tree_records(Ctx *c)
{
    if (c->tree_beta_set == (double)c->tree_beta) return DWG_OK;
    const int64_t nn = (int64_t)2 << c->tree_levels;
    k_tree_records<<<(unsigned)ceil_div(nn, 256), 256, 0, c->stream>>>(
        nn, c->d_tree_A, c->d_tree_C, c->d_tree_R, (double)c->tree_beta, c->d_tree_rec);
    DWG_CUDA_TRY(c, cudaGetLastError());
    c->tree_beta_set = (double)c->tree_beta;
    return DWG_OK;
}

cudaError_t launch_tree_moments(Ctx *c)
{
    const int64_t nleaf = (int64_t)1 << c->tree_levels, nn = 2 * nleaf;
    const int B = 256;
    k_tree_leaf_moments<<<(unsigned)ceil_div(nleaf, B), B, 0, c->stream>>>(
        c->d_p4, c->d_nrm, c->n, nleaf, c->tree_leaf, c->d_tree_M);
    for (int lv = c->tree_levels - 1; lv >= 0; --lv) {
        int64_t first = (int64_t)1 << lv;
        k_tree_level_moments<<<(unsigned)ceil_div(first, B), B, 0, c->stream>>>(first, c->d_tree_M);
    }
    k_tree_moment_records<<<(unsigned)ceil_div(nn, B), B, 0, c->stream>>>(nn, c->d_tree_M,
                                                                           c->d_tree_mrec);
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

cudaError_t launch_tree_gwn(Ctx *c, const float4 *q, int64_t m, bool grad, float *part,
                            int64_t stride, const IterState *st)
{
    EvalParams ep = make_eval_params(c);
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

}  // namespace dwg
