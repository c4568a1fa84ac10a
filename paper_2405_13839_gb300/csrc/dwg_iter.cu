// dwg_iter.cu -- the per-iteration steps after the GWN evaluation
// (paper Alg. 1, Sec. 4.3, Sec. 5.1):
//   k_iso          iso-value w_bar = mean of w over the input points (Eq. 6,
//                  averaged over the inputs), FP64, fixed summation order;
//   k_mc_faces     level set of w - w_bar in every octree leaf, realised as
//                  the six-tetrahedron split of the leaf cube; one face per
//                  cut tetrahedron with its vector area (the cross-product
//                  gradient of Sec. 4.3) oriented toward increasing w;
//   k_knn_scatter  each face adds its vector to its k nearest input points
//                  (Eq. 7); sums are 64-bit fixed point, so the result does
//                  not depend on the order of the atomic additions;
//   k_normal_update  n_i <- -sum / |sum| (a point no face chose keeps its
//                  normal), the per-point change in degrees, next sources;
//   k_sel_*        convergence statistic of Sec. 5.1: mean of the
//                  ceil(n / 100) largest changes, by an exact multi-CTA radix
//                  select on the float bits, then the loop condition.
// and the once-per-cloud steps around it:
//   k_cell_radius, k_cell_lists  per-leaf candidate lists of the faces'
//                  k-nearest search (exact; built once per discretisation);
//   k_init_pca, k_init_gauss     PCA and Gauss-map initial normals (Sec. 5.1);
//   k_voronoi_area              local-Voronoi area weights (Sec. 5.1);
//   k_clamp_delta               clamp radii of the modified kernel (Sec. 5.2);
//   k_mc_tris                   the level set as triangles (the output);
//   k_features                  patch features of the learned warm start.
#include <algorithm>

#include <string.h>

#include "dwg_internal.cuh"

namespace dwg {

// ---------------------------------------------------------------------------
// iso-value
// ---------------------------------------------------------------------------
__device__ __forceinline__ void iso_body(const double *__restrict__ wsum_blocks, int nb,
                                         int64_t n, IterState *st)
{
    if (cloud_idle(st)) return;  // finished cloud of a batch
    __shared__ double sh[256];
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += wsum_blocks[b];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        st->iso = sh[0] / (double)n;
        st->nfaces = 0;
        st->ndefer = 0;
    }
}

__global__ void k_iso(const double *__restrict__ wsum_blocks, int nb, int64_t n, IterState *st)
{
    iso_body(wsum_blocks, nb, n, st);
}

// ---------------------------------------------------------------------------
// level-set faces
// ---------------------------------------------------------------------------
__constant__ int c_tets[6][4] = {{0, 1, 3, 7}, {0, 3, 2, 7}, {0, 2, 6, 7},
                                 {0, 6, 4, 7}, {0, 4, 5, 7}, {0, 5, 1, 7}};

struct F3 {
    float x, y, z;
};
__device__ __forceinline__ F3 f3(float4 v) { return {v.x, v.y, v.z}; }
__device__ __forceinline__ F3 operator-(F3 a, F3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ F3 cross(F3 a, F3 b)
{
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ F3 lerp0(F3 xa, float fa, F3 xb, float fb)
{
    float t = fa / (fa - fb);
    return {xa.x + t * (xb.x - xa.x), xa.y + t * (xb.y - xa.y), xa.z + t * (xb.z - xa.z)};
}

// polygon of one tetrahedron: returns false when the level set misses it
__device__ __forceinline__ bool tet_face(const F3 x[4], const float f[4], const bool ab[4],
                                         F3 &area, F3 &cen)
{
    int na = (int)ab[0] + (int)ab[1] + (int)ab[2] + (int)ab[3];
    if (na == 0 || na == 4) return false;
    F3 P[4];
    int np;
    if (na == 1 || na == 3) {
        bool want = (na == 1);
        int lone = 0;
        for (int i = 0; i < 4; ++i)
            if (ab[i] == want) lone = i;
        np = 0;
        for (int i = 0; i < 4; ++i)
            if (i != lone) P[np++] = lerp0(x[lone], f[lone], x[i], f[i]);
        area = cross(P[1] - P[0], P[2] - P[0]);
    } else {
        int a0 = -1, a1 = -1, b0 = -1, b1 = -1;
        for (int i = 0; i < 4; ++i) {
            if (ab[i]) { if (a0 < 0) a0 = i; else a1 = i; }
            else { if (b0 < 0) b0 = i; else b1 = i; }
        }
        P[0] = lerp0(x[a0], f[a0], x[b0], f[b0]);
        P[1] = lerp0(x[a0], f[a0], x[b1], f[b1]);
        P[2] = lerp0(x[a1], f[a1], x[b1], f[b1]);
        P[3] = lerp0(x[a1], f[a1], x[b0], f[b0]);
        np = 4;
        area = cross(P[2] - P[0], P[3] - P[1]);
    }
    area.x *= 0.5f; area.y *= 0.5f; area.z *= 0.5f;
    F3 ca = {0, 0, 0}, cb = {0, 0, 0};
    for (int i = 0; i < 4; ++i) {
        if (ab[i]) { ca.x += x[i].x; ca.y += x[i].y; ca.z += x[i].z; }
        else { cb.x += x[i].x; cb.y += x[i].y; cb.z += x[i].z; }
    }
    float ia = 1.f / na, ib = 1.f / (4 - na);
    F3 dir = {ca.x * ia - cb.x * ib, ca.y * ia - cb.y * ib, ca.z * ia - cb.z * ib};
    if (area.x * dir.x + area.y * dir.y + area.z * dir.z < 0.f) {
        area.x = -area.x; area.y = -area.y; area.z = -area.z;
    }
    F3 s = {0, 0, 0};
    for (int i = 0; i < np; ++i) { s.x += P[i].x; s.y += P[i].y; s.z += P[i].z; }
    float inv = 1.f / np;
    cen = {s.x * inv, s.y * inv, s.z * inv};
    return true;
}

// Triangles of one tetrahedron's piece of the level set (0, 1 or 2), on the
// same edge points as tet_face, wound so that (v1 - v0) x (v2 - v0) points
// toward decreasing w (outward for outward normals).
__device__ __forceinline__ int tet_tris(const F3 x[4], const float f[4], const bool ab[4],
                                        F3 T[2][3])
{
    int na = (int)ab[0] + (int)ab[1] + (int)ab[2] + (int)ab[3];
    if (na == 0 || na == 4) return 0;
    F3 P[4];
    int nt;
    if (na == 1 || na == 3) {
        bool want = (na == 1);
        int lone = 0;
        for (int i = 0; i < 4; ++i)
            if (ab[i] == want) lone = i;
        int np = 0;
        for (int i = 0; i < 4; ++i)
            if (i != lone) P[np++] = lerp0(x[lone], f[lone], x[i], f[i]);
        T[0][0] = P[0]; T[0][1] = P[1]; T[0][2] = P[2];
        nt = 1;
    } else {
        int a0 = -1, a1 = -1, b0 = -1, b1 = -1;
        for (int i = 0; i < 4; ++i) {
            if (ab[i]) { if (a0 < 0) a0 = i; else a1 = i; }
            else { if (b0 < 0) b0 = i; else b1 = i; }
        }
        P[0] = lerp0(x[a0], f[a0], x[b0], f[b0]);  // a cycle of the quad
        P[1] = lerp0(x[a0], f[a0], x[b1], f[b1]);
        P[2] = lerp0(x[a1], f[a1], x[b1], f[b1]);
        P[3] = lerp0(x[a1], f[a1], x[b0], f[b0]);
        T[0][0] = P[0]; T[0][1] = P[1]; T[0][2] = P[2];
        T[1][0] = P[0]; T[1][1] = P[2]; T[1][2] = P[3];
        nt = 2;
    }
    F3 ca = {0, 0, 0}, cb = {0, 0, 0};
    for (int i = 0; i < 4; ++i) {
        if (ab[i]) { ca.x += x[i].x; ca.y += x[i].y; ca.z += x[i].z; }
        else { cb.x += x[i].x; cb.y += x[i].y; cb.z += x[i].z; }
    }
    float ia = 1.f / na, ib = 1.f / (4 - na);
    F3 down = {cb.x * ib - ca.x * ia, cb.y * ib - ca.y * ia, cb.z * ib - ca.z * ia};
    F3 nrm = nt == 1 ? cross(P[1] - P[0], P[2] - P[0]) : cross(P[2] - P[0], P[3] - P[1]);
    if (nrm.x * down.x + nrm.y * down.y + nrm.z * down.z < 0.f)
        for (int t = 0; t < nt; ++t) {
            F3 v = T[t][1];
            T[t][1] = T[t][2];
            T[t][2] = v;
        }
    return nt;
}

// The level set as triangles: the same corner values and decisions as
// k_mc_faces.  Without FILL only the count; with FILL each leaf writes its
// triangles (9 floats) at an index from the counter, those below cap.
template <bool FILL>
__global__ void __launch_bounds__(256)
    k_mc_tris(const int *__restrict__ leaf_corners, int64_t nl, const float4 *__restrict__ cpos,
              const float *__restrict__ wc, const IterState *st, float *__restrict__ out,
              int64_t cap, unsigned long long *counter)
{
    int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nl) return;
    const double iso = st->iso;
    F3 x[8];
    float f[8];
    bool ab[8];
    for (int v = 0; v < 8; ++v) {
        int ci = leaf_corners[l * 8 + v];
        x[v] = f3(cpos[ci]);
        double df = (double)wc[ci] - iso;
        f[v] = (float)df;
        ab[v] = df > 0.0;
    }
    F3 T[12][3];
    int nt = 0;
#pragma unroll
    for (int t = 0; t < 6; ++t) {
        F3 xt[4];
        float ft[4];
        bool at[4];
        for (int i = 0; i < 4; ++i) {
            int v = c_tets[t][i];
            xt[i] = x[v];
            ft[i] = f[v];
            at[i] = ab[v];
        }
        F3 tt[2][3];
        const int k = tet_tris(xt, ft, at, tt);
        for (int j = 0; j < k; ++j) {
            T[nt][0] = tt[j][0];
            T[nt][1] = tt[j][1];
            T[nt][2] = tt[j][2];
            ++nt;
        }
    }
    if (nt == 0) return;
    const unsigned long long base = atomicAdd(counter, (unsigned long long)nt);
    if (!FILL) return;
    for (int j = 0; j < nt; ++j) {
        const unsigned long long o = base + j;
        if (o >= (unsigned long long)cap) break;
        float *r = out + 9 * o;
        for (int v = 0; v < 3; ++v) {
            r[3 * v + 0] = T[j][v].x;
            r[3 * v + 1] = T[j][v].y;
            r[3 * v + 2] = T[j][v].z;
        }
    }
}

cudaError_t launch_mc_tris(Ctx *c, float *out, int64_t cap, unsigned long long *counter)
{
    const unsigned g = (unsigned)ceil_div(c->nleaves, 256);
    if (out)
        k_mc_tris<true><<<g, 256, 0, c->stream>>>(c->d_leaf_corners, c->nleaves, c->d_corner_pos,
                                                  c->d_wc, c->d_state, out, cap, counter);
    else
        k_mc_tris<false><<<g, 256, 0, c->stream>>>(c->d_leaf_corners, c->nleaves,
                                                   c->d_corner_pos, c->d_wc, c->d_state, nullptr,
                                                   0, counter);
    return cudaGetLastError();
}

// Faces of the level set.  Each face record also carries its leaf's index
// (in the area's w) and, in the centroid's w, the position in the
// Morton-sorted points of the face's leaf cell (found once per cut leaf):
// the k-nearest search of its faces starts there.
__device__ __forceinline__ void mc_faces_body(const int *__restrict__ leaf_corners,
                                              const int4 *__restrict__ leaves, int64_t nl,
                                              const float4 *__restrict__ cpos,
                                              const float *__restrict__ wc,
                                              const uint64_t *__restrict__ codes, int64_t n,
                                              IterState *st, float4 *__restrict__ faces,
                                              int64_t max_faces, int *err, int64_t bid)
{
    if (cloud_idle(st)) return;  // finished cloud of a batch
    int64_t l = bid * blockDim.x + threadIdx.x;
    const double iso = st->iso;
    F3 area[6], cen[6];
    int cnt = 0;
    if (l < nl) {
        F3 x[8];
        float f[8];
        bool ab[8];
        for (int v = 0; v < 8; ++v) {
            int ci = leaf_corners[l * 8 + v];
            x[v] = f3(cpos[ci]);
            double df = (double)wc[ci] - iso;
            f[v] = (float)df;
            ab[v] = df > 0.0;
        }
#pragma unroll
        for (int t = 0; t < 6; ++t) {
            F3 xt[4];
            float ft[4];
            bool at[4];
            for (int i = 0; i < 4; ++i) {
                int v = c_tets[t][i];
                xt[i] = x[v];
                ft[i] = f[v];
                at[i] = ab[v];
            }
            if (tet_face(xt, ft, at, area[cnt], cen[cnt])) ++cnt;
        }
    }
    int seed = 0;
    if (cnt > 0) {
        const int4 L = leaves[l];
        const uint64_t code = ((uint64_t)(uint32_t)L.y | ((uint64_t)(uint32_t)L.z << 32))
                              << (3 * (kMortonBits - L.x));
        int64_t lo = 0, hi = n;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (__ldg(&codes[mid]) < code) lo = mid + 1; else hi = mid;
        }
        seed = (int)lo;
    }
    // warp-aggregated append
    const int lane = threadIdx.x & 31;
    int incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    int total = __shfl_sync(0xffffffffu, incl, 31);
    int base = 0;
    if (lane == 31 && total > 0) base = atomicAdd(&st->nfaces, total);
    base = __shfl_sync(0xffffffffu, base, 31);
    int64_t o = (int64_t)base + incl - cnt;
    for (int k = 0; k < cnt; ++k, ++o) {
        if (o >= max_faces) {
            atomicOr(err, kErrOverflow);
            break;
        }
        faces[2 * o] = make_float4(area[k].x, area[k].y, area[k].z, __int_as_float((int)l));
        faces[2 * o + 1] = make_float4(cen[k].x, cen[k].y, cen[k].z, __int_as_float(seed));
    }
}

__global__ void __launch_bounds__(256)
    k_mc_faces(const int *__restrict__ leaf_corners, const int4 *__restrict__ leaves, int64_t nl,
               const float4 *__restrict__ cpos, const float *__restrict__ wc,
               const uint64_t *__restrict__ codes, int64_t n, IterState *st,
               float4 *__restrict__ faces, int64_t max_faces, int *err)
{
    mc_faces_body(leaf_corners, leaves, nl, cpos, wc, codes, n, st, faces, max_faces, err,
                  blockIdx.x);
}

// ---------------------------------------------------------------------------
// exact k nearest points over the bucket tree
// ---------------------------------------------------------------------------
__device__ __forceinline__ float box_d2(float4 lo, float4 hi, F3 q)
{
    float dx = fmaxf(fmaxf(lo.x - q.x, q.x - hi.x), 0.f);
    float dy = fmaxf(fmaxf(lo.y - q.y, q.y - hi.y), 0.f);
    float dz = fmaxf(fmaxf(lo.z - q.z, q.z - hi.z), 0.f);
    return fmaf(dz, dz, fmaf(dy, dy, __fmul_rn(dx, dx)));
}
__device__ __forceinline__ float pt_d2(float4 p, F3 q)
{
    float dx = __fsub_rn(p.x, q.x), dy = __fsub_rn(p.y, q.y), dz = __fsub_rn(p.z, q.z);
    return fmaf(dz, dz, fmaf(dy, dy, __fmul_rn(dx, dx)));
}

// Candidate order: squared float32 distance, ties to the smaller input index,
// as one 64-bit key (the bits of a non-negative float order like the float).
__device__ __forceinline__ uint64_t knn_key(float d, int64_t o)
{
    return ((uint64_t)__float_as_uint(d) << 32) | (uint64_t)(uint32_t)o;
}

template <int KMAX, bool FIXED>
__device__ __forceinline__ void knn_insert(uint64_t key, int j, int k, uint64_t *best, int *bj)
{
#pragma unroll
    for (int t = KMAX - 1; t >= 0; --t) {
        if (!FIXED && t >= k) continue;
        bool prev = t > 0 && key < best[t > 0 ? t - 1 : 0];
        bool cur = key < best[t];
        if (prev) {
            best[t] = best[t - 1];
            bj[t] = bj[t - 1];
        } else if (cur) {
            best[t] = key;
            bj[t] = j;
        }
    }
}

// Exact k nearest points of q.  KMAX is the array size; with FIXED the
// runtime k equals KMAX and every index is a compile-time constant (the
// arrays stay in registers).  The list is seeded with the points next to q's
// Morton code in the sorted order, which bounds the search ball before the
// depth-first descent (nearer child first) prunes the bucket tree.
// With budget >= 0 the search gives up after that many node visits and
// point distances, returns false and leaves in *bound the k-th smallest
// distance (squared) found so far: an upper bound of q's k-th nearest.
template <int KMAX, bool FIXED>
__device__ __forceinline__ bool knn_search(const KnnTree &T, F3 q, int k, int *bj, int *err,
                                           int64_t seed = -1, int budget = -1,
                                           float *bound = nullptr)
{
    uint64_t best[KMAX];
#pragma unroll
    for (int t = 0; t < KMAX; ++t) {
        best[t] = ~0ull;
        bj[t] = -1;
    }
    const int kk = FIXED ? KMAX : k;
    // seed: the sorted neighbours of q's position on the Morton curve (or a
    // given position near q)
    int64_t lo = seed;
    if (lo < 0) {
        uint64_t code = morton3((uint64_t)quant21(q.x, T.cube_lo[0], T.inv_h21),
                                (uint64_t)quant21(q.y, T.cube_lo[1], T.inv_h21),
                                (uint64_t)quant21(q.z, T.cube_lo[2], T.inv_h21));
        int64_t hi = T.n;
        lo = 0;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (__ldg(&T.codes[mid]) < code) lo = mid + 1; else hi = mid;
        }
    }
    const int64_t s0 = max((int64_t)0, lo - kk), s1 = min(T.n, lo + kk);
    for (int64_t j = s0; j < s1; ++j) {
        float d = pt_d2(__ldg(&T.p4[j]), q);
        uint64_t key = knn_key(d, __ldg(&T.perm[j]));
        if (key < best[kk - 1]) knn_insert<KMAX, FIXED>(key, (int)j, k, best, bj);
    }
    const int64_t nleaf = (int64_t)1 << T.levels;
    int stack[64];
    int sp = 0;
    int work = 0;
    stack[sp++] = 1;
    while (sp > 0) {
        int node = stack[--sp];
        const float worst = best[kk - 1] == ~0ull ? INFINITY : __uint_as_float((uint32_t)(best[kk - 1] >> 32));
        if (budget >= 0 && work > budget) {
            *bound = worst;
            return false;
        }
        ++work;
        if (box_d2(__ldg(&T.lo[node]), __ldg(&T.hi[node]), q) > worst) continue;
        if (node >= nleaf) {
            int64_t j0 = (int64_t)(node - nleaf) * kBucket;
            int64_t j1 = min(j0 + kBucket, T.n);
            work += (int)(j1 - j0);
            for (int64_t j = j0; j < j1; ++j) {
                if (j >= s0 && j < s1) continue;  // already seeded
                float d = pt_d2(__ldg(&T.p4[j]), q);
                if (d > worst) continue;
                uint64_t key = knn_key(d, __ldg(&T.perm[j]));
                if (key < best[kk - 1]) knn_insert<KMAX, FIXED>(key, (int)j, k, best, bj);
            }
        } else {
            int a = 2 * node, b = 2 * node + 1;
            float da = box_d2(__ldg(&T.lo[a]), __ldg(&T.hi[a]), q);
            float db = box_d2(__ldg(&T.lo[b]), __ldg(&T.hi[b]), q);
            if (sp + 2 > 64) {
                atomicOr(err, kErrStack);
                break;
            }
            // push the farther child first so that the nearer one is visited first
            if (da <= db) {
                if (db <= worst) stack[sp++] = b;
                if (da <= worst) stack[sp++] = a;
            } else {
                if (da <= worst) stack[sp++] = a;
                if (db <= worst) stack[sp++] = b;
            }
        }
    }
    return true;
}

// The k nearest of q among a candidate list that is known to contain them:
// the same keys and insertion as knn_search, so the same result.
template <int KMAX, bool FIXED>
__device__ __forceinline__ void knn_scan(const KnnTree &T, F3 q, int k, const int *__restrict__ cand,
                                         int64_t c0, int64_t c1, int *bj)
{
    uint64_t best[KMAX];
#pragma unroll
    for (int t = 0; t < KMAX; ++t) {
        best[t] = ~0ull;
        bj[t] = -1;
    }
    const int kk = FIXED ? KMAX : k;
    float worst = INFINITY;
    for (int64_t t = c0; t < c1; ++t) {
        const int j = __ldg(&cand[t]);
        const float d = pt_d2(__ldg(&T.p4[j]), q);
        if (d > worst) continue;  // the tie-break index is only needed from here
        const uint64_t key = knn_key(d, __ldg(&T.perm[j]));
        if (key < best[kk - 1]) {
            knn_insert<KMAX, FIXED>(key, j, k, best, bj);
            if (best[kk - 1] != ~0ull) worst = __uint_as_float((uint32_t)(best[kk - 1] >> 32));
        }
    }
}

static KnnTree knn_tree(const Ctx *c);

// The scatter's additions are first summed per warp in a shared-memory
// table keyed by point (open addressing, a few probes), then each distinct
// point of the warp takes one global addition per component.  Neighbouring
// faces share most of their nearest points, and where the level set lies
// away from the points many faces share the same few; summing them in the
// warp first keeps the global atomics few and uncontended.  A table per warp
// (not per block) lets each warp leave as soon as its own faces are done.
// The sums are 64-bit fixed-point integers, so the grouping changes no bit.
// The tables take 28 KB of shared memory per block, which the SM takes from
// its L1 cache: on clouds of millions of points the searches' gathers lose
// more to the smaller cache than the tables save (a 3M-point union: 80.8 ->
// 40.7 ms with them; a 15M-point union: 49 -> 70 ms), so clouds above
// kAggMaxPoints add straight to the points' sums.
constexpr int kAggBits = 8;
constexpr int kAggSlots = 1 << kAggBits;  // table entries per warp of 32 faces
constexpr int kAggWarps = 4;              // warps of a 128-thread block
constexpr int kAggProbes = 8;    // entries tried before adding to global memory directly
constexpr int64_t kAggMaxPoints = 4000000;
constexpr size_t kAggSmem =
    (size_t)kAggWarps * kAggSlots * (3 * sizeof(unsigned long long) + sizeof(int));

// A face whose own search (no candidate list for its cell) runs past
// kSearchBudget -- a face far from the points, about as far from many of
// them, as near the centre of a sphere -- is deferred: its index and the
// bound its partial search reached go to a list that k_knn_deferred finishes
// with a whole block per face, so that no single thread holds the launch.
template <int KMAX, bool FIXED>
__device__ __forceinline__ void knn_scatter_body(const float4 *__restrict__ faces,
                                                 IterState *st, int64_t max_faces,
                                                 const KnnTree &T, int k,
                                                 const int64_t *__restrict__ cell_off,
                                                 const int *__restrict__ cell_idx, double scale,
                                                 unsigned long long *acc, int2 *defer,
                                                 int budget, bool agg, int *err, int64_t bid)
{
    if (cloud_idle(st)) return;  // finished cloud of a batch
    const int64_t nf = min((int64_t)st->nfaces, max_faces);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (bid * blockDim.x + wid * 32 >= nf) return;  // the whole warp is past the faces
    // agg: kAggSmem bytes of dynamic shared memory, per warp 3 x kAggSlots
    // sums, then every warp's kAggSlots keys
    extern __shared__ unsigned long long s_agg[];
    unsigned long long *s_v = s_agg + (size_t)wid * 3 * kAggSlots;
    int *s_key = reinterpret_cast<int *>(s_agg + (size_t)kAggWarps * 3 * kAggSlots) +
                 wid * kAggSlots;
    if (agg) {
        for (int i = lane; i < kAggSlots; i += 32) {
            s_key[i] = -1;
            s_v[i] = s_v[kAggSlots + i] = s_v[2 * kAggSlots + i] = 0ull;
        }
    }
    const int64_t f = bid * blockDim.x + threadIdx.x;
    const bool active = f < nf;
    int bj[KMAX];
#pragma unroll
    for (int t = 0; t < KMAX; ++t) bj[t] = -1;
    long long vx = 0, vy = 0, vz = 0;
    if (active) {
        float4 A = faces[2 * f], C = faces[2 * f + 1];
        int64_t c0 = 0, c1 = 0;
        if (cell_off) {
            const int leaf = __float_as_int(A.w);
            c0 = __ldg(&cell_off[leaf]);
            c1 = __ldg(&cell_off[leaf + 1]);
        }
        if (c1 > c0) {
            knn_scan<KMAX, FIXED>(T, F3{C.x, C.y, C.z}, k, cell_idx, c0, c1, bj);
        } else {
            // one inlined search: budgeted first, unbounded when the list is full
            const F3 q{C.x, C.y, C.z};
            const int64_t seed = (int64_t)__float_as_int(C.w);
            int bud = budget;
            float bound = INFINITY;
            while (!knn_search<KMAX, FIXED>(T, q, k, bj, err, seed, bud, &bound)) {
                const int slot = atomicAdd(&st->ndefer, 1);
                if (slot < kDeferCap) {
                    defer[slot] = make_int2((int)f, __float_as_int(bound));
#pragma unroll
                    for (int t = 0; t < KMAX; ++t) bj[t] = -1;  // added by k_knn_deferred
                    break;
                }
                bud = -1;
            }
        }
        vx = llrint((double)A.x * scale);
        vy = llrint((double)A.y * scale);
        vz = llrint((double)A.z * scale);
    }
    if (!agg) {  // straight to the points' sums
#pragma unroll
        for (int t = 0; t < KMAX; ++t) {
            if (t >= k || bj[t] < 0) continue;
            unsigned long long *a = acc + 3 * (int64_t)bj[t];
            atomicAdd(a + 0, (unsigned long long)vx);
            atomicAdd(a + 1, (unsigned long long)vy);
            atomicAdd(a + 2, (unsigned long long)vz);
        }
        return;
    }
    __syncwarp();  // the table is cleared
#pragma unroll
    for (int t = 0; t < KMAX; ++t) {
        if (t >= k || bj[t] < 0) continue;
        const int j = bj[t];
        unsigned h = ((unsigned)j * 2654435761u) >> (32 - kAggBits);
        bool added = false;
        for (int p = 0; p < kAggProbes; ++p, h = (h + 1) & (kAggSlots - 1)) {
            const int prev = atomicCAS(&s_key[h], -1, j);
            if (prev == -1 || prev == j) {
                atomicAdd(&s_v[h], (unsigned long long)vx);
                atomicAdd(&s_v[kAggSlots + h], (unsigned long long)vy);
                atomicAdd(&s_v[2 * kAggSlots + h], (unsigned long long)vz);
                added = true;
                break;
            }
        }
        if (!added) {  // the table is crowded: straight to the point's sums
            unsigned long long *a = acc + 3 * (int64_t)j;
            atomicAdd(a + 0, (unsigned long long)vx);
            atomicAdd(a + 1, (unsigned long long)vy);
            atomicAdd(a + 2, (unsigned long long)vz);
        }
    }
    __syncwarp();  // every addition is in the table
    for (int i = lane; i < kAggSlots; i += 32) {
        const int j = s_key[i];
        if (j < 0) continue;
        unsigned long long *a = acc + 3 * (int64_t)j;
        atomicAdd(a + 0, s_v[i]);
        atomicAdd(a + 1, s_v[kAggSlots + i]);
        atomicAdd(a + 2, s_v[2 * kAggSlots + i]);
    }
}

// 8 resident blocks per SM (64 registers): the search is a chain of
// dependent loads that wants the warps
template <int KMAX, bool FIXED>
__global__ void __launch_bounds__(128, KMAX > 16 ? 1 : 8)
    k_knn_scatter(const float4 *__restrict__ faces, IterState *st, int64_t max_faces,
                  KnnTree T, int k, const int64_t *__restrict__ cell_off,
                  const int *__restrict__ cell_idx, double scale, unsigned long long *acc,
                  int2 *defer, int budget, int agg, int *err)
{
    knn_scatter_body<KMAX, FIXED>(faces, st, max_faces, T, k, cell_off, cell_idx, scale, acc,
                                  defer, budget, agg != 0, err, blockIdx.x);
}

// The deferred faces, one block per face (the blocks take the list in
// turn; 128 threads for k <= 16, 64 for up to 32 so that the lists fit the
// static shared memory).  The threads first test the bucket tree's nodes at
// one level of at most 2,048 nodes against the bound of the face's partial
// search (an upper bound of its k-th nearest distance), then split the
// buckets under the nodes that pass, skipping buckets whose box lies beyond
// the bound; each thread keeps its own k nearest under the search's
// (distance, input index) keys; thread 0 takes the k smallest of the
// block's lists -- the k points the full search finds -- and adds the
// face's vector to them.
template <int KMAX>
__host__ __device__ constexpr int defer_threads() { return KMAX > 16 ? 64 : 128; }

template <int KMAX, bool FIXED>
__device__ __forceinline__ void knn_deferred_body(const float4 *__restrict__ faces,
                                                  const IterState *st,
                                                  const int2 *__restrict__ defer,
                                                  const KnnTree &T, int k, double scale,
                                                  unsigned long long *acc, int64_t bid,
                                                  int64_t nblk)
{
    if (cloud_idle(st)) return;  // finished cloud of a batch
    const int nd = min(st->ndefer, kDeferCap);
    if (bid >= nd) return;  // the same for every thread of the block
    constexpr int NT = defer_threads<KMAX>();
    __shared__ uint64_t s_key[NT * KMAX];
    __shared__ int s_j[NT * KMAX];
    __shared__ int s_head[NT];
    constexpr int kCoarseBits = 11;
    __shared__ int s_pass[1 << kCoarseBits];
    __shared__ int s_npass;
    const int kk = FIXED ? KMAX : k;
    const int64_t nleaf = (int64_t)1 << T.levels;
    const int64_t nb = (T.n + kBucket - 1) / kBucket;
    const int lc = min(T.levels, kCoarseBits);      // the coarse level
    const int64_t span = (int64_t)1 << (T.levels - lc);  // buckets under a coarse node
    for (int64_t d = bid; d < nd; d += nblk) {
        const int2 e = defer[d];
        const int64_t f = e.x;
        const float4 C = faces[2 * f + 1];
        const F3 q{C.x, C.y, C.z};
        uint64_t best[KMAX];
        int bj[KMAX];
#pragma unroll
        for (int t = 0; t < KMAX; ++t) {
            best[t] = ~0ull;
            bj[t] = -1;
        }
        float worst = __int_as_float(e.y);
        if (threadIdx.x == 0) s_npass = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < (1 << lc); i += NT) {
            const int node = (1 << lc) + i;
            if ((int64_t)i * span < nb &&
                box_d2(__ldg(&T.lo[node]), __ldg(&T.hi[node]), q) <= worst)
                s_pass[atomicAdd(&s_npass, 1)] = i;
        }
        __syncthreads();
        const int64_t total = (int64_t)s_npass * span;
        for (int64_t u = threadIdx.x; u < total; u += NT) {
            const int64_t b = (int64_t)s_pass[u / span] * span + u % span;
            if (b >= nb) continue;
            const int64_t node = nleaf + b;
            if (box_d2(__ldg(&T.lo[node]), __ldg(&T.hi[node]), q) > worst) continue;
            const int64_t j0 = b * kBucket, j1 = min(j0 + kBucket, T.n);
            for (int64_t j = j0; j < j1; ++j) {
                const float d2 = pt_d2(__ldg(&T.p4[j]), q);
                if (d2 > worst) continue;
                const uint64_t key = knn_key(d2, __ldg(&T.perm[j]));
                if (key < best[kk - 1]) {
                    knn_insert<KMAX, FIXED>(key, (int)j, k, best, bj);
                    if (best[kk - 1] != ~0ull)
                        worst = fminf(worst, __uint_as_float((uint32_t)(best[kk - 1] >> 32)));
                }
            }
        }
#pragma unroll
        for (int t = 0; t < KMAX; ++t) {
            s_key[threadIdx.x * KMAX + t] = best[t];
            s_j[threadIdx.x * KMAX + t] = bj[t];
        }
        s_head[threadIdx.x] = 0;
        __syncthreads();
        if (threadIdx.x == 0) {
            const float4 A = faces[2 * f];
            const long long vx = llrint((double)A.x * scale);
            const long long vy = llrint((double)A.y * scale);
            const long long vz = llrint((double)A.z * scale);
            for (int r = 0; r < kk; ++r) {  // the r-th smallest key of the block
                uint64_t m = ~0ull;
                int win = -1;
                for (int t = 0; t < NT; ++t) {
                    const int hd = s_head[t];
                    if (hd < kk && s_key[t * KMAX + hd] < m) {
                        m = s_key[t * KMAX + hd];
                        win = t;
                    }
                }
                if (win < 0 || m == ~0ull) break;  // fewer than k points
                const int j = s_j[win * KMAX + s_head[win]];
                s_head[win] += 1;
                unsigned long long *a = acc + 3 * (int64_t)j;
                atomicAdd(a + 0, (unsigned long long)vx);
                atomicAdd(a + 1, (unsigned long long)vy);
                atomicAdd(a + 2, (unsigned long long)vz);
            }
        }
        __syncthreads();  // the lists are read before the next face reuses them
    }
}

template <int KMAX, bool FIXED>
__global__ void __launch_bounds__(defer_threads<KMAX>())
    k_knn_deferred(const float4 *__restrict__ faces, const IterState *st,
                   const int2 *__restrict__ defer, KnnTree T, int k, double scale,
                   unsigned long long *acc)
{
    knn_deferred_body<KMAX, FIXED>(faces, st, defer, T, k, scale, acc, blockIdx.x, gridDim.x);
}

template <int KMAX, bool FIXED>
__global__ void k_knn_query(const float4 *__restrict__ q, int64_t m, KnnTree T, int k,
                            int64_t *idx_out, int *err)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    float4 v = q[i];
    int bj[KMAX];
    knn_search<KMAX, FIXED>(T, F3{v.x, v.y, v.z}, k, bj, err);
    for (int t = 0; t < k; ++t) idx_out[i * k + t] = bj[t] >= 0 ? T.perm[bj[t]] : -1;
}

// distance from each of m sampled points (sorted indices, strided) to its
// 11th nearest point (itself included: the 10th nearest other point)
__global__ void k_spacing(KnnTree T, int64_t m, int64_t stride, float *d_out, int *err)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const float4 v = T.p4[min(i * stride, T.n - 1)];
    const F3 q = {v.x, v.y, v.z};
    int bj[11];
    knn_search<11, true>(T, q, 11, bj, err);
    d_out[i] = bj[10] >= 0 ? sqrtf(pt_d2(T.p4[bj[10]], q)) : 0.f;
}

cudaError_t launch_spacing(Ctx *c, int64_t m, float *d_out)
{
    const int64_t stride = std::max<int64_t>(1, c->n / std::max<int64_t>(m, 1));
    k_spacing<<<(unsigned)ceil_div(m, 128), 128, 0, c->stream>>>(knn_tree(c), m, stride, d_out,
                                                                 c->d_err);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// learned warm start: patch features from the 16 nearest other points
// ---------------------------------------------------------------------------
__global__ void k_centroid(const float4 *__restrict__ p4, int64_t n, double *out /* cx,cy,cz,R */)
{
    __shared__ double sh[256][3];
    double s[3] = {0.0, 0.0, 0.0};
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        float4 p = p4[i];
        s[0] += p.x; s[1] += p.y; s[2] += p.z;
    }
    for (int k = 0; k < 3; ++k) sh[threadIdx.x][k] = s[k];
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int k = 0; k < 3; ++k) sh[threadIdx.x][k] += sh[threadIdx.x + o][k];
        __syncthreads();
    }
    const double cx = sh[0][0] / n, cy = sh[0][1] / n, cz = sh[0][2] / n;
    __syncthreads();
    double r = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        float4 p = p4[i];
        double dx = p.x - cx, dy = p.y - cy, dz = p.z - cz;
        r += dx * dx + dy * dy + dz * dz;
    }
    sh[threadIdx.x][0] = r;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x][0] += sh[threadIdx.x + o][0];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = cx;
        out[1] = cy;
        out[2] = cz;
        out[3] = sqrt(sh[0][0] / n);
    }
}

// Feature row of sorted point i: offsets to its 16 nearest other points (in
// ascending order) divided by their RMS length, then (p - c) / R, zero
// padding to 64.  Rows go to row index perm[i] when by_input is set.
__global__ void __launch_bounds__(128)
    k_features(KnnTree T, const double *__restrict__ cR, float *__restrict__ X, int by_input,
               int *err)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= T.n) return;
    const float4 pi = T.p4[i];
    int bj[17];
    knn_search<17, true>(T, F3{pi.x, pi.y, pi.z}, 17, bj, err);
    float o[48];
    int cnt = 0;
    float ss = 0.f;
#pragma unroll
    for (int t = 0; t < 17; ++t) {
        int j = bj[t];
        if (j < 0 || j == (int)i || cnt == 16) continue;
        float4 pj = T.p4[j];
        float dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
        o[3 * cnt] = dx;
        o[3 * cnt + 1] = dy;
        o[3 * cnt + 2] = dz;
        ss += dx * dx + dy * dy + dz * dz;
        ++cnt;
    }
    float s = cnt > 0 ? sqrtf(ss / cnt) : 0.f;
    float inv = s > 0.f ? 1.f / s : 0.f;
    float *row = X + (by_input ? T.perm[i] : i) * 64;
    for (int k = 0; k < 48; ++k) row[k] = k < 3 * cnt ? o[k] * inv : 0.f;
    double R = cR[3];
    row[48] = R > 0.0 ? (float)((pi.x - cR[0]) / R) : 0.f;
    row[49] = R > 0.0 ? (float)((pi.y - cR[1]) / R) : 0.f;
    row[50] = R > 0.0 ? (float)((pi.z - cR[2]) / R) : 0.f;
    for (int k = 51; k < 64; ++k) row[k] = 0.f;
}

// network outputs (sorted order) -> unit initial normals; an output that is
// zero or not finite keeps the random normal already in nrm
__global__ void k_normals_from_y(const float *__restrict__ Y, int64_t n, float4 *nrm)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float x = Y[3 * i], y = Y[3 * i + 1], z = Y[3 * i + 2];
    float l = sqrtf(x * x + y * y + z * z);
    if (l > 1e-12f && isfinite(l)) nrm[i] = make_float4(x / l, y / l, z / l, 0.f);
}

cudaError_t launch_features(Ctx *c, float *X, bool by_input, double *cR)
{
    k_centroid<<<1, 256, 0, c->stream>>>(c->d_p4, c->n, cR);
    k_features<<<(unsigned)ceil_div(c->n, 128), 128, 0, c->stream>>>(knn_tree(c), cR, X,
                                                                      by_input ? 1 : 0, c->d_err);
    return cudaGetLastError();
}

cudaError_t launch_normals_from_y(Ctx *c, const float *Y)
{
    k_normals_from_y<<<(unsigned)ceil_div(c->n, 256), 256, 0, c->stream>>>(Y, c->n, c->d_nrm);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// PCA and Gauss-map initial normals (Sec. 5.1, "Normal Initialization")
// ---------------------------------------------------------------------------
// Unit eigenvector of the smallest eigenvalue of the symmetric 3 x 3 matrix a
// (destroyed), by cyclic Jacobi rotations: each rotation is the symmetric
// 2 x 2 Schur decomposition of Golub and Van Loan (Matrix Computations,
// Sec. 8.5) applied to the (p, q) plane.  False for the zero matrix or a
// non-finite result.
__device__ bool sym3_min_eigvec(double a[3][3], double out[3])
{
    double fro = 0.0;
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k) fro += a[r][k] * a[r][k];
    if (!(fro > 0.0) || !isfinite(fro)) return false;
    double v[3][3] = {{1.0, 0.0, 0.0}, {0.0, 1.0, 0.0}, {0.0, 0.0, 1.0}};
    for (int sweep = 0; sweep < 16; ++sweep) {
        const double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
        if (off <= 1e-36 * fro) break;  // off-diagonal below double rounding of the entries
        for (int r = 0; r < 3; ++r) {
            const int p = r == 2 ? 1 : 0, q = r == 0 ? 1 : 2;  // (0,1), (0,2), (1,2)
            if (a[p][q] == 0.0) continue;
            const double tau = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
            // A <- J^T A J and V <- V J, J the identity but for J_pp = J_qq = c,
            // J_pq = s, J_qp = -s
            for (int k = 0; k < 3; ++k) {
                const double x = a[k][p], y = a[k][q];
                a[k][p] = c * x - s * y;
                a[k][q] = s * x + c * y;
            }
            for (int k = 0; k < 3; ++k) {
                const double x = a[p][k], y = a[q][k];
                a[p][k] = c * x - s * y;
                a[q][k] = s * x + c * y;
            }
            for (int k = 0; k < 3; ++k) {
                const double x = v[k][p], y = v[k][q];
                v[k][p] = c * x - s * y;
                v[k][q] = s * x + c * y;
            }
        }
    }
    int m = 0;
    if (a[1][1] < a[m][m]) m = 1;
    if (a[2][2] < a[m][m]) m = 2;
    const double l = sqrt(v[0][m] * v[0][m] + v[1][m] * v[1][m] + v[2][m] * v[2][m]);
    if (!(l > 0.0) || !isfinite(l)) return false;
    for (int k = 0; k < 3; ++k) out[k] = v[k][m] / l;
    return true;
}

// PCA normal of sorted point i: the smallest-eigenvalue eigenvector of the
// covariance of its kPcaK nearest points (itself included), in FP64 on the
// offsets from p_i.  PCA fixes the line only; the direction is the one away
// from the bounding-box centre c (the Gauss-map side, n . (p_i - c) > 0),
// and +z, then +y, then +x where that dot product is zero.  Where the
// covariance is zero the random normal already in nrm stays.
__global__ void __launch_bounds__(128)
    k_init_pca(KnnTree T, double cx, double cy, double cz, float4 *__restrict__ nrm, int *err)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= T.n) return;
    const float4 pi = T.p4[i];
    int bj[kPcaK];
    knn_search<kPcaK, true>(T, F3{pi.x, pi.y, pi.z}, kPcaK, bj, err);
    double d[kPcaK][3], mean[3] = {0.0, 0.0, 0.0};
    int cnt = 0;
#pragma unroll
    for (int t = 0; t < kPcaK; ++t) {
        if (bj[t] < 0) continue;
        const float4 pj = T.p4[bj[t]];
        d[cnt][0] = (double)pj.x - (double)pi.x;
        d[cnt][1] = (double)pj.y - (double)pi.y;
        d[cnt][2] = (double)pj.z - (double)pi.z;
        for (int k = 0; k < 3; ++k) mean[k] += d[cnt][k];
        ++cnt;
    }
    if (cnt < 1) return;
    for (int k = 0; k < 3; ++k) mean[k] /= cnt;
    double C[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
    for (int t = 0; t < cnt; ++t) {
        const double e0 = d[t][0] - mean[0], e1 = d[t][1] - mean[1], e2 = d[t][2] - mean[2];
        C[0][0] += e0 * e0; C[0][1] += e0 * e1; C[0][2] += e0 * e2;
        C[1][1] += e1 * e1; C[1][2] += e1 * e2; C[2][2] += e2 * e2;
    }
    C[1][0] = C[0][1]; C[2][0] = C[0][2]; C[2][1] = C[1][2];
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k) C[r][k] /= cnt;
    double e[3];
    if (!sym3_min_eigvec(C, e)) return;
    const double side = e[0] * ((double)pi.x - cx) + e[1] * ((double)pi.y - cy) +
                        e[2] * ((double)pi.z - cz);
    const bool flip = side != 0.0
                          ? side < 0.0
                          : (e[2] < 0.0 || (e[2] == 0.0 && (e[1] < 0.0 || (e[1] == 0.0 && e[0] < 0.0))));
    const double sg = flip ? -1.0 : 1.0;
    nrm[i] = make_float4((float)(sg * e[0]), (float)(sg * e[1]), (float)(sg * e[2]), 0.f);
}

// Gauss-map normal: the direction from the bounding-box centre c to p_i, in
// FP64; a point at c keeps its random normal.
__global__ void k_init_gauss(const float4 *__restrict__ p4, int64_t n, double cx, double cy,
                             double cz, float4 *__restrict__ nrm)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 p = p4[i];
    const double dx = (double)p.x - cx, dy = (double)p.y - cy, dz = (double)p.z - cz;
    const double l = sqrt(dx * dx + dy * dy + dz * dz);
    if (l > 0.0) nrm[i] = make_float4((float)(dx / l), (float)(dy / l), (float)(dz / l), 0.f);
}

cudaError_t launch_init_pca(Ctx *c)
{
    k_init_pca<<<(unsigned)ceil_div(c->n, 128), 128, 0, c->stream>>>(
        knn_tree(c), c->bbox_c[0], c->bbox_c[1], c->bbox_c[2], c->d_nrm, c->d_err);
    return cudaGetLastError();
}

cudaError_t launch_init_gauss(Ctx *c)
{
    k_init_gauss<<<(unsigned)ceil_div(c->n, 256), 256, 0, c->stream>>>(
        c->d_p4, c->n, c->bbox_c[0], c->bbox_c[1], c->bbox_c[2], c->d_nrm);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// local-Voronoi area weights (Sec. 5.1, "Computing Area Weights")
// ---------------------------------------------------------------------------
// A convex polygon of k vertices (counter-clockwise) clipped by the
// half-plane ax x + ay y <= b; at most cap output vertices (a convex polygon
// gains at most one per clip; *over is set if rounding asked for more).
__device__ int vor_clip(const double *px, const double *py, int k, double ax, double ay, double b,
                        double *ox, double *oy, int cap, bool *over)
{
    int o = 0;
    for (int t = 0; t < k; ++t) {
        const int u = t + 1 == k ? 0 : t + 1;
        const double fp = ax * px[t] + ay * py[t] - b, fq = ax * px[u] + ay * py[u] - b;
        if (fp <= 0.0) {
            if (o < cap) { ox[o] = px[t]; oy[o] = py[t]; ++o; } else *over = true;
        }
        if ((fp < 0.0 && fq > 0.0) || (fq < 0.0 && fp > 0.0)) {
            const double s = fp / (fp - fq);
            if (o < cap) {
                ox[o] = px[t] + s * (px[u] - px[t]);
                oy[o] = py[t] + s * (py[u] - py[t]);
                ++o;
            } else {
                *over = true;
            }
        }
    }
    return o;
}

// Area of a convex polygon containing the origin intersected with the disk of
// radius R about the origin: each edge (A, B) spans the triangle (0, A, B);
// the part of the edge inside the circle adds its triangle, the parts outside
// add circular sectors R^2 * angle / 2.
__device__ double vor_disk_area(const double *px, const double *py, int k, double R)
{
    double total = 0.0;
    const double R2 = R * R;
    for (int t = 0; t < k; ++t) {
        const int u = t + 1 == k ? 0 : t + 1;
        const double ax = px[t], ay = py[t], dx = px[u] - ax, dy = py[u] - ay;
        const double a = dx * dx + dy * dy, b = ax * dx + ay * dy, c = ax * ax + ay * ay - R2;
        if (a == 0.0) continue;
        const double disc = b * b - a * c;
        double s1 = 0.0, s2 = 0.0;
        if (disc > 0.0) {
            const double r = sqrt(disc);
            s1 = fmin(fmax((-b - r) / a, 0.0), 1.0);
            s2 = fmin(fmax((-b + r) / a, 0.0), 1.0);
        }
        const double x1 = ax + s1 * dx, y1 = ay + s1 * dy, x2 = ax + s2 * dx, y2 = ay + s2 * dy;
        const double bx = px[u], by = py[u];
        // no crossing: s1 = s2 = 0, one sector from A to B
        total += 0.5 * R2 * atan2(ax * y1 - ay * x1, ax * x1 + ay * y1);
        total += 0.5 * (x1 * y2 - y1 * x2);
        total += 0.5 * R2 * atan2(x2 * by - y2 * bx, x2 * bx + y2 * by);
    }
    return total;
}

// Cell area of sorted point i: its m nearest other points, the PCA tangent
// plane through it, the projected neighbours as Voronoi seeds, the cell of
// the origin cut to the disk of half the largest projected distance.  A
// neighbourhood with no extent gives 0 (the caller substitutes the mean).
template <int KMAX, bool FIXED>
__global__ void __launch_bounds__(128)
    k_voronoi_area(KnnTree T, int m, double *__restrict__ area, int *err)
{
    constexpr int CAP = KMAX + 4;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= T.n) return;
    const float4 pi = T.p4[i];
    int bj[KMAX];
    knn_search<KMAX, FIXED>(T, F3{pi.x, pi.y, pi.z}, m + 1, bj, err);
    double d[KMAX][3];
    double mean[3] = {0.0, 0.0, 0.0};
    int cnt = 0;
#pragma unroll
    for (int t = 0; t < KMAX; ++t) {
        const int j = bj[t];
        if (t > m || j < 0 || j == (int)i || cnt == m) continue;
        const float4 pj = T.p4[j];
        d[cnt][0] = (double)pj.x - (double)pi.x;
        d[cnt][1] = (double)pj.y - (double)pi.y;
        d[cnt][2] = (double)pj.z - (double)pi.z;
        for (int k = 0; k < 3; ++k) mean[k] += d[cnt][k];
        ++cnt;
    }
    area[i] = 0.0;
    if (cnt < 1) return;
    for (int k = 0; k < 3; ++k) mean[k] /= (cnt + 1);  // p_i itself is the zero offset
    double C[3][3];
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k) C[r][k] = mean[r] * mean[k];  // the zero offset's term
    for (int t = 0; t < cnt; ++t)
        for (int r = 0; r < 3; ++r)
            for (int k = 0; k < 3; ++k) C[r][k] += (d[t][r] - mean[r]) * (d[t][k] - mean[k]);
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k) C[r][k] /= (cnt + 1);
    double nv[3];
    if (!sym3_min_eigvec(C, nv)) return;
    // tangent basis: e1 = normalise(n x axis least aligned with n), e2 = n x e1
    int ax = 0;
    if (fabs(nv[1]) < fabs(nv[ax])) ax = 1;
    if (fabs(nv[2]) < fabs(nv[ax])) ax = 2;
    double e1[3] = {ax == 2 ? nv[1] : (ax == 1 ? -nv[2] : 0.0),
                    ax == 0 ? nv[2] : (ax == 2 ? -nv[0] : 0.0),
                    ax == 1 ? nv[0] : (ax == 0 ? -nv[1] : 0.0)};
    const double l1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    for (int k = 0; k < 3; ++k) e1[k] /= l1;
    const double e2[3] = {nv[1] * e1[2] - nv[2] * e1[1], nv[2] * e1[0] - nv[0] * e1[2],
                          nv[0] * e1[1] - nv[1] * e1[0]};
    double qx[KMAX], qy[KMAX], R = 0.0;
    for (int t = 0; t < cnt; ++t) {
        qx[t] = d[t][0] * e1[0] + d[t][1] * e1[1] + d[t][2] * e1[2];
        qy[t] = d[t][0] * e2[0] + d[t][1] * e2[1] + d[t][2] * e2[2];
        R = fmax(R, sqrt(qx[t] * qx[t] + qy[t] * qy[t]));
    }
    R *= 0.5;
    if (!(R > 0.0)) return;
    double ax0[CAP], ay0[CAP], ax1[CAP], ay1[CAP];
    ax0[0] = -R; ay0[0] = -R; ax0[1] = R; ay0[1] = -R;
    ax0[2] = R;  ay0[2] = R;  ax0[3] = -R; ay0[3] = R;
    int k = 4;
    bool over = false;
    for (int t = 0; t < cnt && k >= 3; ++t) {
        const double r2 = qx[t] * qx[t] + qy[t] * qy[t];
        if (!(r2 > 0.0)) continue;  // a seed on the origin imposes nothing
        k = vor_clip(ax0, ay0, k, qx[t], qy[t], 0.5 * r2, ax1, ay1, CAP, &over);
        for (int v = 0; v < k; ++v) {
            ax0[v] = ax1[v];
            ay0[v] = ay1[v];
        }
    }
    if (over) atomicOr(err, kErrGeometry);
    if (k >= 3) area[i] = vor_disk_area(ax0, ay0, k, R);
}

// mean of the positive areas (one block, fixed order)
__global__ void k_area_mean(const double *__restrict__ area, int64_t n, double *out)
{
    __shared__ double ss[256];
    __shared__ double sc[256];
    double s = 0.0, c = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
        if (area[i] > 0.0) { s += area[i]; c += 1.0; }
    ss[threadIdx.x] = s;
    sc[threadIdx.x] = c;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            ss[threadIdx.x] += ss[threadIdx.x + o];
            sc[threadIdx.x] += sc[threadIdx.x + o];
        }
        __syncthreads();
    }
    // no positive area at all (a cloud of one point, or all copies of one):
    // the paper's default weight 1
    if (threadIdx.x == 0) out[0] = sc[0] > 0.0 ? ss[0] / sc[0] : 1.0;
}

// install a_i (zero areas take the mean) into p4.w; optionally write them in
// input order
__global__ void k_area_install(const double *__restrict__ area, const double *__restrict__ mean,
                               const int64_t *__restrict__ perm, int64_t n, float4 *p4,
                               float *a_out, int *err)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double a = area[i] > 0.0 ? area[i] : mean[0];
    const float f = (float)a;
    if (!(f > 0.f) || !isfinite(f)) atomicOr(err, kErrNonfinite);
    p4[i].w = f;
    if (a_out) a_out[perm[i]] = f;
}

cudaError_t launch_voronoi_weights(Ctx *c, int m, double *scratch /* n + 1 */, float *a_out)
{
    const unsigned g = (unsigned)ceil_div(c->n, 128);
    if (m == 15)
        k_voronoi_area<16, true><<<g, 128, 0, c->stream>>>(knn_tree(c), m, scratch, c->d_err);
    else
        k_voronoi_area<32, false><<<g, 128, 0, c->stream>>>(knn_tree(c), m, scratch, c->d_err);
    k_area_mean<<<1, 256, 0, c->stream>>>(scratch, c->n, scratch + c->n);
    k_area_install<<<(unsigned)ceil_div(c->n, 256), 256, 0, c->stream>>>(
        scratch, scratch + c->n, c->d_perm, c->n, c->d_p4, a_out, c->d_err);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// clamp radii of the modified Poisson kernel (Sec. 5.2, "Poisson Kernels")
// ---------------------------------------------------------------------------
// delta_i = mean distance (FP64) from p_i to those of its k nearest other
// points whose distance lies in [vmin, vmax]; if none does, the mean of all
// k distances clamped to [vmin, vmax].  Stored as delta^2 in float32 (sorted
// order) and, when asked, delta in input order.
template <int KMAX, bool FIXED>
__global__ void __launch_bounds__(128)
    k_clamp_delta(KnnTree T, int k, double vmin, double vmax, float *__restrict__ delta2,
                  float *__restrict__ delta_out, int *err)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= T.n) return;
    const float4 pi = T.p4[i];
    int bj[KMAX];
    knn_search<KMAX, FIXED>(T, F3{pi.x, pi.y, pi.z}, k + 1, bj, err);
    double sum_in = 0.0, sum_all = 0.0;
    int n_in = 0, cnt = 0;
#pragma unroll
    for (int t = 0; t < KMAX; ++t) {
        const int j = bj[t];
        if (t > k || j < 0 || j == (int)i || cnt == k) continue;
        const float4 pj = T.p4[j];
        const double dx = (double)pj.x - (double)pi.x, dy = (double)pj.y - (double)pi.y,
                     dz = (double)pj.z - (double)pi.z;
        const double d = sqrt(dx * dx + dy * dy + dz * dz);
        sum_all += d;
        ++cnt;
        if (d >= vmin && d <= vmax) {
            sum_in += d;
            ++n_in;
        }
    }
    double delta = vmin;
    if (n_in > 0) delta = sum_in / n_in;
    else if (cnt > 0) delta = fmin(fmax(sum_all / cnt, vmin), vmax);
    delta2[i] = (float)(delta * delta);
    if (delta_out) delta_out[T.perm[i]] = (float)delta;
}

cudaError_t launch_clamp_delta(Ctx *c, int k, double vmin, double vmax, float *delta_out)
{
    const unsigned g = (unsigned)ceil_div(c->n, 128);
    if (k == 10)
        k_clamp_delta<11, true><<<g, 128, 0, c->stream>>>(knn_tree(c), k, vmin, vmax, c->d_delta2,
                                                           delta_out, c->d_err);
    else
        k_clamp_delta<32, false><<<g, 128, 0, c->stream>>>(knn_tree(c), k, vmin, vmax,
                                                            c->d_delta2, delta_out, c->d_err);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// normal update (Eq. 7) and per-point change
// ---------------------------------------------------------------------------
__device__ __forceinline__ void normal_update_body(int mode, int64_t n,
                                                   unsigned long long *__restrict__ acc,
                                                   const float4 *__restrict__ wg,
                                                   const float4 *__restrict__ p4,
                                                   float4 *__restrict__ nrm,
                                                   float *__restrict__ src,
                                                   float *__restrict__ src16,
                                                   float *__restrict__ dtheta,
                                                   double *__restrict__ dn_blocks,
                                                   const IterState *st, int64_t bid)
{
    if (cloud_idle(st)) return;  // finished cloud of a batch: normals stay
    int64_t i = bid * blockDim.x + threadIdx.x;
    double dn = 0.0;
    if (i < n) {
        float4 o = nrm[i];
        float nx = o.x, ny = o.y, nz = o.z;
        if (mode == DWG_UPDATE_LEVELSET) {
            // -sum / |sum| does not depend on the fixed-point scale: the
            // integer sums go to float (relative rounding 2^-24) and are
            // normalised in FP32 (FP64 runs at a small fraction of FP32 here)
            unsigned long long *a = acc + 3 * i;
            const float ax = __ll2float_rn((long long)a[0]);
            const float ay = __ll2float_rn((long long)a[1]);
            const float az = __ll2float_rn((long long)a[2]);
            a[0] = 0ull; a[1] = 0ull; a[2] = 0ull;
            const float len = sqrtf(fmaf(az, az, fmaf(ay, ay, ax * ax)));
            if (len > 0.f && isfinite(len)) {
                nx = -ax / len;
                ny = -ay / len;
                nz = -az / len;
            }
        } else {
            float4 g = wg[i];
            float len = sqrtf(g.x * g.x + g.y * g.y + g.z * g.z);
            if (len > 0.f && isfinite(len)) {
                nx = -g.x / len;
                ny = -g.y / len;
                nz = -g.z / len;
            }
        }
        float cx = o.y * nz - o.z * ny, cy = o.z * nx - o.x * nz, cz = o.x * ny - o.y * nx;
        float sn = sqrtf(cx * cx + cy * cy + cz * cz);
        float cs = o.x * nx + o.y * ny + o.z * nz;
        dtheta[i] = atan2f(sn, cs) * (float)(180.0 / kPi);
        float ex = nx - o.x, ey = ny - o.y, ez = nz - o.z;
        dn = (double)sqrtf(ex * ex + ey * ey + ez * ez);
        nrm[i] = make_float4(nx, ny, nz, 0.f);
        float c = p4[i].w * (float)(1.0 / (4.0 * kPi));
        float mx = c * nx, my = c * ny, mz = c * nz;
        // only the moment words of the record change: (mx, mx) as one 8-byte
        // store (no read of the position words), then (my, my, mz, mz)
        float *r = src + i * kSrcFloats;
        *reinterpret_cast<float2 *>(r + 6) = make_float2(mx, mx);
        *reinterpret_cast<float4 *>(r + 8) = make_float4(my, my, mz, mz);
        if (src16) {  // the modified kernel's records (same first 12 floats)
            float *r16 = src16 + i * kSrcFloatsClamp;
            *reinterpret_cast<float2 *>(r16 + 6) = make_float2(mx, mx);
            *reinterpret_cast<float4 *>(r16 + 8) = make_float4(my, my, mz, mz);
        }
    }
    __shared__ double sh[256];
    sh[threadIdx.x] = dn;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) dn_blocks[bid] = sh[0];
}

__global__ void __launch_bounds__(256)
    k_normal_update(int mode, int64_t n, unsigned long long *__restrict__ acc,
                    const float4 *__restrict__ wg, const float4 *__restrict__ p4,
                    float4 *__restrict__ nrm, float *__restrict__ src,
                    float *__restrict__ src16, float *__restrict__ dtheta,
                    double *__restrict__ dn_blocks, const IterState *st)
{
    normal_update_body(mode, n, acc, wg, p4, nrm, src, src16, dtheta, dn_blocks, st, blockIdx.x);
}

// ---------------------------------------------------------------------------
// convergence: exact mean of the ceil(n/100) largest changes
// ---------------------------------------------------------------------------
constexpr int kSelThreads = 1024;

// exclusive block scan of one unsigned per thread (1024 threads)
__device__ unsigned block_scan_u(unsigned v, unsigned *warp_sums, unsigned &total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        unsigned x = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += x;
    }
    if (lane == 31) warp_sums[w] = incl;
    __syncthreads();
    if (w == 0) {
        unsigned s = warp_sums[lane];
        unsigned si = s;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned x = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) si += x;
        }
        warp_sums[lane] = si - s;
        if (lane == 31) warp_sums[32] = si;
    }
    __syncthreads();
    unsigned r = warp_sums[w] + incl - v;
    total = warp_sums[32];
    __syncthreads();
    return r;
}

// Among the bins of hist (nb bins, 4 per thread), find b with
// suffix(b) >= k > suffix(b + 1); returns b and the count strictly above.
__device__ void find_bin(const unsigned *hist, int nb, unsigned k, unsigned *warp_sums,
                         int *s_bin, unsigned *s_above)
{
    unsigned loc[4];
    unsigned s = 0;
    int b0 = threadIdx.x * 4;
    for (int t = 0; t < 4; ++t) {
        loc[t] = (b0 + t < nb) ? hist[b0 + t] : 0u;
        s += loc[t];
    }
    unsigned total;
    unsigned ex = block_scan_u(s, warp_sums, total);
    for (int t = 0; t < 4; ++t) {
        int b = b0 + t;
        unsigned suffix = total - ex;  // count in bins >= b
        if (b < nb && suffix >= k && suffix - loc[t] < k) {
            *s_bin = b;
            *s_above = suffix - loc[t];
        }
        ex += loc[t];
    }
    __syncthreads();
}

// The exact k-th largest change by a three-level radix select on the float
// bits (non-negative floats order like their bit patterns): bits 31..20,
// 19..8, 7..0.  Each level is a histogram over all changes by many CTAs
// (shared-memory bins, then integer atomics into the global bins: exact)
// and one CTA that finds the bin holding the k-th largest; then a grid sums
// the changes strictly above the threshold into per-block FP64 partials
// and one CTA adds the partials in a fixed order and takes the decision.
constexpr int kSelGridThreads = 256;

__device__ __forceinline__ void sel_hist_body(const float *__restrict__ dtheta, int64_t n,
                                              int level, const SelState *__restrict__ ss,
                                              unsigned *__restrict__ hist, const IterState *st,
                                              int64_t bid, int64_t nblk)
{
    if (cloud_idle(st)) return;
    __shared__ unsigned h[kSelBins];
    for (int b = threadIdx.x; b < kSelBins; b += blockDim.x) h[b] = 0;
    __syncthreads();
    const unsigned *bits = reinterpret_cast<const unsigned *>(dtheta);
    const int shift = level == 0 ? 20 : (level == 1 ? 8 : 0);
    const unsigned mask = level == 2 ? 255u : 4095u;
    const int sh_hi = level == 1 ? 20 : 8;  // bits above this level's field (levels 1, 2)
    const unsigned prefix = ss->prefix;
    for (int64_t i = bid * blockDim.x + threadIdx.x; i < n; i += nblk * blockDim.x) {
        const unsigned v = bits[i];
        if (level > 0 && (v >> sh_hi) != prefix) continue;
        atomicAdd(&h[(v >> shift) & mask], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kSelBins; b += blockDim.x)
        if (h[b]) atomicAdd(&hist[b], h[b]);
}

__global__ void __launch_bounds__(kSelGridThreads)
    k_sel_hist(const float *__restrict__ dtheta, int64_t n, int level,
               const SelState *__restrict__ ss, unsigned *__restrict__ hist, const IterState *st)
{
    sel_hist_body(dtheta, n, level, ss, hist, st, blockIdx.x, gridDim.x);
}

__device__ __forceinline__ void sel_find_body(int64_t n, int level, SelState *__restrict__ ss,
                                              unsigned *__restrict__ hist, const IterState *st)
{
    if (cloud_idle(st)) return;
    __shared__ unsigned warp_sums[33];
    __shared__ int s_bin;
    __shared__ unsigned s_above;
    const int nb = level == 2 ? 256 : 4096;
    if (level == 0 && threadIdx.x == 0) {
        ss->krem = (unsigned)((n + 99) / 100);
        ss->above = 0;
        ss->prefix = 0;
    }
    __syncthreads();
    find_bin(hist, nb, ss->krem, warp_sums, &s_bin, &s_above);
    if (threadIdx.x == 0) {
        ss->prefix = (ss->prefix << (level == 2 ? 8 : 12)) | (unsigned)s_bin;
        ss->above += s_above;
        ss->krem -= s_above;
    }
    for (int b = threadIdx.x; b < kSelBins; b += blockDim.x) hist[b] = 0;  // for the next level
}

__global__ void __launch_bounds__(kSelThreads)
    k_sel_find(int64_t n, int level, SelState *__restrict__ ss, unsigned *__restrict__ hist,
               const IterState *st)
{
    sel_find_body(n, level, ss, hist, st);
}

__device__ __forceinline__ void sel_sum_body(const float *__restrict__ dtheta, int64_t n,
                                             const SelState *__restrict__ ss,
                                             double *__restrict__ part, const IterState *st,
                                             int64_t bid, int64_t nblk)
{
    if (cloud_idle(st)) return;
    __shared__ double sh[kSelGridThreads];
    const unsigned *bits = reinterpret_cast<const unsigned *>(dtheta);
    const unsigned tbits = ss->prefix;
    double s = 0.0;
    for (int64_t i = bid * blockDim.x + threadIdx.x; i < n; i += nblk * blockDim.x)
        if (bits[i] > tbits) s += (double)dtheta[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[bid] = sh[0];
}

__global__ void __launch_bounds__(kSelGridThreads)
    k_sel_sum(const float *__restrict__ dtheta, int64_t n, const SelState *__restrict__ ss,
              double *__restrict__ part, const IterState *st)
{
    sel_sum_body(dtheta, n, ss, part, st, blockIdx.x, gridDim.x);
}

__device__ __forceinline__ void sel_final_body(int64_t n, float tol, int rule,
                                               const SelState *__restrict__ ss,
                                               const double *__restrict__ part, int npart,
                                               IterState *st,
                                               const double *__restrict__ dn_blocks, int ndn,
                                               double *tr_iso, double *tr_stat, double *tr_dn,
                                               long long *tr_faces,
                                               cudaGraphConditionalHandle cond, int use_cond)
{
    if (cloud_idle(st)) return;  // finished cloud of a batch
    __shared__ double sh[kSelThreads];
    double s = 0.0;
    for (int b = threadIdx.x; b < npart; b += blockDim.x) s += part[b];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    const double sum_above = sh[0];
    __syncthreads();
    double dn = 0.0;
    for (int b = threadIdx.x; b < ndn; b += blockDim.x) dn += dn_blocks[b];
    sh[threadIdx.x] = dn;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const unsigned k = (unsigned)((n + 99) / 100);
        const float tval = __uint_as_float(ss->prefix);
        double stat = (sum_above + (double)(k - ss->above) * (double)tval) / (double)k;
        int it = st->iter;
        st->stat = stat;
        if (tr_iso && it < st->max_iters) {
            tr_iso[it] = st->iso;
            tr_stat[it] = stat;
            tr_dn[it] = sh[0] / (double)n;
            tr_faces[it] = st->nfaces;
        }
        it += 1;
        st->iter = it;
        // rule 0: mean of the largest 1 % of the changes <= tol degrees (Sec. 5.1);
        // rule 1: mean |n_new - n_old| over all points <= 2 sin(tol / 2), the
        // chord of tol degrees (the measure plotted in Fig. 6)
        const double chord = 2.0 * sin((double)tol * (kPi / 360.0));
        int done = rule == 1 ? (sh[0] / (double)n <= chord) : (stat <= (double)tol);
        st->done = done;
        if (use_cond) cudaGraphSetConditional(cond, (!done && it < st->max_iters) ? 1u : 0u);
    }
}

__global__ void __launch_bounds__(kSelThreads)
    k_sel_final(int64_t n, float tol, int rule, const SelState *__restrict__ ss,
                const double *__restrict__ part, int npart, IterState *st,
                const double *__restrict__ dn_blocks, int ndn, double *tr_iso, double *tr_stat,
                double *tr_dn, long long *tr_faces, cudaGraphConditionalHandle cond, int use_cond)
{
    sel_final_body(n, tol, rule, ss, part, npart, st, dn_blocks, ndn, tr_iso, tr_stat, tr_dn,
                   tr_faces, cond, use_cond);
}

// ---------------------------------------------------------------------------
// random unit normals from splitmix64 (stream 7)
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_random_normals(float4 *nrm, const int64_t *perm, int64_t n, uint64_t key)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t j = (uint64_t)perm[i];
    const uint64_t G = 0x9E3779B97F4A7C15ull;
    uint64_t a = mix64(key + (2 * j + 1) * G), b = mix64(key + (2 * j + 2) * G);
    double u0 = (double)(a >> 11) * 0x1.0p-53, u1 = (double)(b >> 11) * 0x1.0p-53;
    double z = 1.0 - 2.0 * u0;
    double phi = 2.0 * kPi * u1;
    double s = sqrt(fmax(0.0, 1.0 - z * z));
    nrm[i] = make_float4((float)(s * cos(phi)), (float)(s * sin(phi)), (float)z, 0.f);
}

cudaError_t launch_random_normals(float4 *nrm, const int64_t *perm, int64_t n, uint64_t seed,
                                  cudaStream_t s)
{
    uint64_t key = mix64(((seed & 0xFFFFFFFFull) << 32) | 7ull);
    k_random_normals<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(nrm, perm, n, key);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static KnnTree knn_tree(const Ctx *c)
{
    KnnTree T;
    T.p4 = c->d_p4;
    T.perm = c->d_perm;
    T.n = c->n;
    T.lo = c->d_bvh_lo;
    T.hi = c->d_bvh_hi;
    T.levels = c->knn_levels;
    T.codes = c->d_codes;
    for (int k = 0; k < 3; ++k) T.cube_lo[k] = c->cube_lo[k];
    T.inv_h21 = (double)(1 << kMortonBits) / c->cube_L;
    return T;
}

cudaError_t launch_iso(Ctx *c)
{
    k_iso<<<1, 256, 0, c->stream>>>(c->d_wsum_blocks, c->wsum_blocks, c->n, c->d_state);
    return cudaGetLastError();
}

// A cloud's entry of the batched iteration's table: the same arguments its
// own launches pass (launch_reduce_points with the points as queries,
// launch_iso, launch_reduce_w, launch_mc_faces, launch_knn_scatter,
// launch_normal_update, launch_select, launch_tree_moments, the list
// evaluation); valid while the cloud's buffers stay (the batch graph's
// generation covers them).
void fill_cloud_iter(const Ctx *c, CloudIter *o)
{
    memset(o, 0, sizeof *o);
    o->st = c->d_state;
    o->err = c->d_err;
    o->counter = c->d_counter;
    o->n = c->n;
    o->ep = make_eval_params(c);
    o->part_p = c->d_part_p;
    o->nchunks_p = c->nchunks_p;
    o->p4 = c->d_p4;
    o->src = c->d_src;
    o->codes = c->d_codes;
    for (int k = 0; k < 3; ++k) o->cq.lo[k] = c->cube_lo[k];
    o->cq.inv_h21 = (double)(1 << kMortonBits) / c->cube_L;
    o->wg = c->d_wg;
    o->wsum_blocks = c->d_wsum_blocks;
    o->wsum_nb = c->wsum_blocks;
    o->part_c = c->d_part_c;
    o->nchunks_c = c->nchunks_c;
    o->ncorners = c->ncorners;
    o->wc = c->d_wc;
    o->leaf_corners = c->d_leaf_corners;
    o->leaves = c->d_leaves;
    o->nleaves = c->nleaves;
    o->corner_pos = c->d_corner_pos;
    o->faces = c->d_faces;
    o->max_faces = c->max_faces;
    o->defer = c->d_defer;
    o->knn_budget = c->knn_budget;
    o->T = knn_tree(c);
    o->k = c->knn;
    const bool lists = c->knn_lists && c->cells_k == c->knn && c->d_cell_off;
    o->cell_off = lists ? c->d_cell_off : nullptr;
    o->cell_idx = lists ? c->d_cell_idx : nullptr;
    o->acc_scale = c->acc_scale;
    o->acc = c->d_acc;
    o->mode = c->mode;
    o->nrm = c->d_nrm;
    o->nrm_c = c->d_nrm;
    o->src_rw = c->d_src;
    o->dtheta = c->d_dtheta;
    o->dn_blocks = c->d_dn_blocks;
    o->sel = c->d_sel;
    o->sel_hist = c->d_sel_hist;
    o->sel_part = c->d_sel_part;
    o->sel_nb = select_blocks(c->n);
    o->tol = c->tol;
    o->conv_rule = c->conv_rule;
    o->tr_iso = c->d_tr_iso;
    o->tr_stat = c->d_tr_stat;
    o->tr_dn = c->d_tr_dn;
    o->tr_faces = c->d_tr_faces;
    o->tree = use_tree(c) ? 1 : 0;
    o->levels = c->tree_levels;
    o->bucket = c->tree_leaf;
    o->tree_M = c->d_tree_M;
    o->tree_rec = c->d_tree_rec;
    o->tree_mrec = c->d_tree_mrec;
    o->tree_frec = c->d_tree_frec;
    const TreeLists *L[2] = {&c->lists_p, &c->lists_c};
    float *lp[2] = {c->d_part_p, c->d_part_c};
    for (int w = 0; w < 2; ++w) {
        o->lq[w] = L[w]->q;
        o->lm[w] = L[w]->m;
        o->far_off[w] = L[w]->d_far_off;
        o->near_off[w] = L[w]->d_near_off;
        o->item_off[w] = L[w]->d_item_off;
        o->far_ids[w] = L[w]->d_far;
        o->near_ids[w] = L[w]->d_near;
        o->items[w] = L[w]->d_items;
        o->nitems[w] = L[w]->nitems;
        o->ipart[w] = L[w]->d_ipart;
        o->lpart[w] = lp[w];
    }
}

cudaError_t launch_mc_faces(Ctx *c)
{
    k_mc_faces<<<(unsigned)ceil_div(c->nleaves, 256), 256, 0, c->stream>>>(
        c->d_leaf_corners, c->d_leaves, c->nleaves, c->d_corner_pos, c->d_wc, c->d_codes, c->n,
        c->d_state, c->d_faces, c->max_faces, c->d_err);
    return cudaGetLastError();
}

cudaError_t launch_knn_scatter(Ctx *c)
{
    // one thread per possible face; threads past the emitted count exit
    unsigned blocks = (unsigned)ceil_div(c->max_faces, 128);
    KnnTree T = knn_tree(c);
    const bool lists = c->knn_lists && c->cells_k == c->knn && c->d_cell_off;
    const int64_t *off = lists ? c->d_cell_off : nullptr;
    const int *idx = lists ? c->d_cell_idx : nullptr;
    // the per-warp sum tables (dynamic shared memory) on clouds up to
    // kAggMaxPoints; batched clouds always take them
    const int agg = c->n <= kAggMaxPoints ? 1 : 0;
    const size_t smem = agg ? kAggSmem : 0;
    if (c->knn == 10) {
        k_knn_scatter<10, true><<<blocks, 128, smem, c->stream>>>(
            c->d_faces, c->d_state, c->max_faces, T, c->knn, off, idx, c->acc_scale, c->d_acc,
            c->d_defer, c->knn_budget, agg, c->d_err);
        k_knn_deferred<10, true><<<kDeferBlocks, defer_threads<10>(), 0, c->stream>>>(
            c->d_faces, c->d_state, c->d_defer, T, c->knn, c->acc_scale, c->d_acc);
    } else {
        k_knn_scatter<32, false><<<blocks, 128, smem, c->stream>>>(
            c->d_faces, c->d_state, c->max_faces, T, c->knn, off, idx, c->acc_scale, c->d_acc,
            c->d_defer, c->knn_budget, agg, c->d_err);
        k_knn_deferred<32, false><<<kDeferBlocks, defer_threads<32>(), 0, c->stream>>>(
            c->d_faces, c->d_state, c->d_defer, T, c->knn, c->acc_scale, c->d_acc);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// per-leaf candidate lists of the faces' k nearest points
// ---------------------------------------------------------------------------
// A face lies in its leaf cell.  With c' the cell centre rounded to float and
// h' >= |x - c'| for every x of the cell (half-diagonal plus the rounding of
// c' and of a face centroid), the k nearest points of c' lie within r_k(c')
// of c', so within r_k(c') + h' of any x: x's k nearest lie within
// R = r_k(c') + 2 h' of c'.  R is widened by a relative 1e-4 and an absolute
// 2^-17 of the coordinates so that float32 distance rounding cannot drop a
// point; extra candidates cost time, never the result.
constexpr int kCellCap = 256;

__device__ __forceinline__ void cell_centre(int4 L, int d, const KnnTree &T, double cube_L,
                                            F3 &cf, double &hp)
{
    const uint64_t code = (uint64_t)(uint32_t)L.y | ((uint64_t)(uint32_t)L.z << 32);
    const double hd = cube_L / (double)(1ll << d);  // finest cell edge
    const double e = hd * (double)(1ll << (d - L.x)); // this cell's edge
    const double cx = T.cube_lo[0] + (double)(compact3(code) << (d - L.x)) * hd + 0.5 * e;
    const double cy = T.cube_lo[1] + (double)(compact3(code >> 1) << (d - L.x)) * hd + 0.5 * e;
    const double cz = T.cube_lo[2] + (double)(compact3(code >> 2) << (d - L.x)) * hd + 0.5 * e;
    cf = F3{(float)cx, (float)cy, (float)cz};
    const double mag = fabs(cx) + fabs(cy) + fabs(cz) + e;
    hp = 0.5 * e * 1.7320508075688772 + ldexp(mag, -17);
}

template <int KMAX, bool FIXED>
__global__ void __launch_bounds__(128)
    k_cell_radius(const int4 *__restrict__ leaves, int64_t nl, int d, double cube_L, KnnTree T,
                  int k, float *__restrict__ R2, int *err)
{
    int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nl) return;
    F3 cf;
    double hp;
    cell_centre(leaves[l], d, T, cube_L, cf, hp);
    int bj[KMAX];
    knn_search<KMAX, FIXED>(T, cf, k, bj, err);
    const int last = bj[(FIXED ? KMAX : k) - 1];
    if (last < 0) {  // fewer than k points: every point is a candidate
        R2[l] = INFINITY;
        return;
    }
    const double rk = sqrt((double)pt_d2(T.p4[last], cf));
    const double R = (rk + 2.0 * hp) * (1.0 + 1e-4) + ldexp(fabs((double)cf.x) + fabs((double)cf.y) +
                                                             fabs((double)cf.z) + rk, -17);
    R2[l] = __double2float_ru(R * R);
}

// points within the radius (FILL: write them; otherwise count, 0 above the cap)
template <bool FILL>
__global__ void __launch_bounds__(128)
    k_cell_lists(const int4 *__restrict__ leaves, int64_t nl, int d, double cube_L, KnnTree T,
                 const float *__restrict__ R2, const int64_t *__restrict__ off,
                 int *__restrict__ idx, int64_t *__restrict__ cnt, int *err)
{
    int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nl) return;
    int64_t o0 = 0, room = 0;
    if (FILL) {
        o0 = off[l];
        room = off[l + 1] - o0;
        if (room <= 0) return;
    }
    F3 cf;
    double hp;
    cell_centre(leaves[l], d, T, cube_L, cf, hp);
    const float r2 = R2[l];
    const int64_t nleaf = (int64_t)1 << T.levels;
    int stack[64];
    int sp = 0;
    int count = 0;
    bool over = false;
    stack[sp++] = 1;
    while (sp > 0 && !over) {
        const int node = stack[--sp];
        if (box_d2(__ldg(&T.lo[node]), __ldg(&T.hi[node]), cf) > r2) continue;
        if (node >= nleaf) {
            const int64_t j0 = (int64_t)(node - nleaf) * kBucket;
            const int64_t j1 = min(j0 + kBucket, T.n);
            for (int64_t j = j0; j < j1; ++j) {
                if (pt_d2(__ldg(&T.p4[j]), cf) > r2) continue;
                if (FILL) {
                    if (count < room) idx[o0 + count] = (int)j;
                } else if (count == kCellCap) {
                    over = true;
                    break;
                }
                ++count;
            }
        } else {
            if (sp + 2 > 64) {
                atomicOr(err, kErrStack);
                break;
            }
            stack[sp++] = 2 * node + 1;
            stack[sp++] = 2 * node;
        }
    }
    if (!FILL) cnt[l] = over ? 0 : count;
    else if (count != room) atomicOr(err, kErrOverflow);  // the two passes must agree
}

void free_cell_lists(Ctx *c)
{
    cudaFree(c->d_cell_off);
    cudaFree(c->d_cell_idx);
    c->d_cell_off = nullptr;
    c->d_cell_idx = nullptr;
    c->cells_k = 0;
}

int build_cell_lists(Ctx *c)
{
    if (!c->knn_lists || c->nleaves < 1) return DWG_OK;
    if (c->cells_k == c->knn && c->d_cell_off) return DWG_OK;
    free_cell_lists(c);
    ++c->bufgen;  // a captured graph holds the old pointers
    const int64_t nl = c->nleaves;
    const int d = c->built_depth;
    KnnTree T = knn_tree(c);
    float *R2 = nullptr;
    int64_t *cnt = nullptr, *tot = nullptr;
    auto body = [&]() -> int {
        DWG_CUDA_TRY(c, cudaMalloc(&R2, nl * sizeof(float)));
        DWG_CUDA_TRY(c, cudaMalloc(&cnt, nl * sizeof(int64_t)));
        DWG_CUDA_TRY(c, cudaMalloc(&tot, sizeof(int64_t)));
        DWG_CUDA_TRY(c, cudaMalloc(&c->d_cell_off, (nl + 1) * sizeof(int64_t)));
        const unsigned g = (unsigned)ceil_div(nl, 128);
        if (c->knn == 10)
            k_cell_radius<10, true><<<g, 128, 0, c->stream>>>(c->d_leaves, nl, d, c->cube_L, T,
                                                               c->knn, R2, c->d_err);
        else
            k_cell_radius<32, false><<<g, 128, 0, c->stream>>>(c->d_leaves, nl, d, c->cube_L, T,
                                                                c->knn, R2, c->d_err);
        k_cell_lists<false><<<g, 128, 0, c->stream>>>(c->d_leaves, nl, d, c->cube_L, T, R2,
                                                      nullptr, nullptr, cnt, c->d_err);
        int rc = scan_i64(c, cnt, c->d_cell_off, nl, tot);
        if (rc) return rc;
        int64_t total = 0;
        DWG_CUDA_TRY(c, cudaMemcpyAsync(&total, tot, sizeof total, cudaMemcpyDeviceToHost,
                                        c->stream));
        DWG_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        DWG_CUDA_TRY(c, cudaMemcpyAsync(c->d_cell_off + nl, tot, sizeof(int64_t),
                                        cudaMemcpyDeviceToDevice, c->stream));
        // lists only where they fit comfortably (a quarter of the free memory)
        size_t fr = 0, tt = 0;
        cudaMemGetInfo(&fr, &tt);
        if ((size_t)total * sizeof(int) > fr / 4) return DWG_ERR_OOM;
        DWG_CUDA_TRY(c, cudaMalloc(&c->d_cell_idx, std::max<int64_t>(total, 1) * sizeof(int)));
        k_cell_lists<true><<<g, 128, 0, c->stream>>>(c->d_leaves, nl, d, c->cube_L, T, R2,
                                                     c->d_cell_off, c->d_cell_idx, nullptr,
                                                     c->d_err);
        DWG_CUDA_TRY(c, cudaGetLastError());
        DWG_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        c->cells_k = c->knn;
        return DWG_OK;
    };
    int rc = body();
    cudaFree(R2);
    cudaFree(cnt);
    cudaFree(tot);
    if (rc) {
        free_cell_lists(c);  // the tree search serves every face
        if (rc == DWG_ERR_OOM) rc = DWG_OK;
    }
    return rc;
}

cudaError_t launch_knn_query(Ctx *c, const float4 *q, int64_t m, int k, int64_t *idx_out)
{
    KnnTree T = knn_tree(c);
    unsigned blocks = (unsigned)ceil_div(m, 128);
    if (k == 10)
        k_knn_query<10, true><<<blocks, 128, 0, c->stream>>>(q, m, T, k, idx_out, c->d_err);
    else
        k_knn_query<32, false><<<blocks, 128, 0, c->stream>>>(q, m, T, k, idx_out, c->d_err);
    return cudaGetLastError();
}

cudaError_t launch_normal_update(Ctx *c)
{
    k_normal_update<<<(unsigned)ceil_div(c->n, 256), 256, 0, c->stream>>>(
        c->mode, c->n, c->d_acc, c->d_wg, c->d_p4, c->d_nrm, c->d_src,
        c->reg_mode == DWG_REG_CLAMP ? c->d_src16 : nullptr, c->d_dtheta, c->d_dn_blocks,
        c->d_state);
    return cudaGetLastError();
}

int select_blocks(int64_t n)
{
    return (int)std::min<int64_t>(std::max<int64_t>(ceil_div(n, 4 * kSelGridThreads), 1), 1024);
}

cudaError_t launch_select(Ctx *c, cudaGraphConditionalHandle cond, int use_cond)
{
    const int nb = select_blocks(c->n);
    for (int level = 0; level < 3; ++level) {
        k_sel_hist<<<nb, kSelGridThreads, 0, c->stream>>>(c->d_dtheta, c->n, level, c->d_sel,
                                                          c->d_sel_hist, c->d_state);
        k_sel_find<<<1, kSelThreads, 0, c->stream>>>(c->n, level, c->d_sel, c->d_sel_hist,
                                                     c->d_state);
    }
    k_sel_sum<<<nb, kSelGridThreads, 0, c->stream>>>(c->d_dtheta, c->n, c->d_sel, c->d_sel_part,
                                                     c->d_state);
    k_sel_final<<<1, kSelThreads, 0, c->stream>>>(
        c->n, c->tol, c->conv_rule, c->d_sel, c->d_sel_part, nb, c->d_state, c->d_dn_blocks,
        (int)ceil_div(c->n, 256), c->d_tr_iso, c->d_tr_stat, c->d_tr_dn, c->d_tr_faces, cond,
        use_cond);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// batched iteration phases: every cloud of a batch in one launch (each
// cloud's blocks as in its own launch, so its results are the same bits)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_iso_b(const CloudIter *__restrict__ cl)
{
    const CloudIter &c = cl[blockIdx.x];
    iso_body(c.wsum_blocks, c.wsum_nb, c.n, c.st);
}

__global__ void __launch_bounds__(256)
    k_mc_faces_b(const CloudIter *__restrict__ cl, const int *__restrict__ off, int ncl)
{
    const int ci = seg_cloud(off, ncl);
    const CloudIter &c = cl[ci];
    mc_faces_body(c.leaf_corners, c.leaves, c.nleaves, c.corner_pos, c.wc, c.codes, c.n, c.st,
                  c.faces, c.max_faces, c.err, (int64_t)blockIdx.x - off[ci]);
}

template <int KMAX, bool FIXED>
__global__ void __launch_bounds__(128)
    k_knn_scatter_b(const CloudIter *__restrict__ cl, const int *__restrict__ off, int ncl)
{
    const int ci = seg_cloud(off, ncl);
    const CloudIter &c = cl[ci];
    knn_scatter_body<KMAX, FIXED>(c.faces, c.st, c.max_faces, c.T, c.k, c.cell_off, c.cell_idx,
                                  c.acc_scale, c.acc, c.defer, c.knn_budget, true, c.err,
                                  (int64_t)blockIdx.x - off[ci]);
}

__global__ void __launch_bounds__(defer_threads<10>())
    k_knn_deferred_b(const CloudIter *__restrict__ cl, const int *__restrict__ off, int ncl)
{
    const int ci = seg_cloud(off, ncl);
    const CloudIter &c = cl[ci];
    knn_deferred_body<10, true>(c.faces, c.st, c.defer, c.T, c.k, c.acc_scale, c.acc,
                                (int64_t)blockIdx.x - off[ci], (int64_t)(off[ci + 1] - off[ci]));
}

__global__ void __launch_bounds__(256)
    k_normal_update_b(const CloudIter *__restrict__ cl, const int *__restrict__ off, int ncl)
{
    const int ci = seg_cloud(off, ncl);
    const CloudIter &c = cl[ci];
    normal_update_body(c.mode, c.n, c.acc, c.wg, c.p4, c.nrm, c.src_rw, nullptr, c.dtheta,
                       c.dn_blocks, c.st, (int64_t)blockIdx.x - off[ci]);
}

__global__ void __launch_bounds__(kSelGridThreads)
    k_sel_hist_b(const CloudIter *__restrict__ cl, const int *__restrict__ off, int ncl, int level)
{
    const int ci = seg_cloud(off, ncl);
    const CloudIter &c = cl[ci];
    sel_hist_body(c.dtheta, c.n, level, c.sel, c.sel_hist, c.st, (int64_t)blockIdx.x - off[ci],
                  (int64_t)off[ci + 1] - off[ci]);
}

__global__ void __launch_bounds__(kSelThreads) k_sel_find_b(const CloudIter *__restrict__ cl, int level)
{
    const CloudIter &c = cl[blockIdx.x];
    sel_find_body(c.n, level, c.sel, c.sel_hist, c.st);
}

__global__ void __launch_bounds__(kSelGridThreads)
    k_sel_sum_b(const CloudIter *__restrict__ cl, const int *__restrict__ off, int ncl)
{
    const int ci = seg_cloud(off, ncl);
    const CloudIter &c = cl[ci];
    sel_sum_body(c.dtheta, c.n, c.sel, c.sel_part, c.st, (int64_t)blockIdx.x - off[ci],
                 (int64_t)off[ci + 1] - off[ci]);
}

__global__ void __launch_bounds__(kSelThreads) k_sel_final_b(const CloudIter *__restrict__ cl)
{
    const CloudIter &c = cl[blockIdx.x];
    sel_final_body(c.n, c.tol, c.conv_rule, c.sel, c.sel_part, c.sel_nb, c.st, c.dn_blocks,
                   (int)((c.n + 255) / 256), c.tr_iso, c.tr_stat, c.tr_dn, c.tr_faces, 0, 0);
}

cudaError_t launch_iter_batch(int phase, const CloudIter *cl, const int *off, int ncl,
                              int blocks, int arg, cudaStream_t s)
{
    if (blocks <= 0) return cudaSuccess;
    const unsigned g = (unsigned)blocks;
    switch (phase) {
    case kPhIso: k_iso_b<<<(unsigned)ncl, 256, 0, s>>>(cl); break;
    case kPhMcFaces: k_mc_faces_b<<<g, 256, 0, s>>>(cl, off, ncl); break;
    case kPhKnn: k_knn_scatter_b<10, true><<<g, 128, kAggSmem, s>>>(cl, off, ncl); break;
    case kPhKnnDefer:
        k_knn_deferred_b<<<g, defer_threads<10>(), 0, s>>>(cl, off, ncl);
        break;
    case kPhUpdate: k_normal_update_b<<<g, 256, 0, s>>>(cl, off, ncl); break;
    case kPhSelHist: k_sel_hist_b<<<g, kSelGridThreads, 0, s>>>(cl, off, ncl, arg); break;
    case kPhSelFind: k_sel_find_b<<<(unsigned)ncl, kSelThreads, 0, s>>>(cl, arg); break;
    case kPhSelSum: k_sel_sum_b<<<g, kSelGridThreads, 0, s>>>(cl, off, ncl); break;
    case kPhSelFinal: k_sel_final_b<<<(unsigned)ncl, kSelThreads, 0, s>>>(cl); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace dwg
