// dwg_build.cu -- position-only structures, built once per cloud:
//   * NaN/Inf check and bounding box of the float32 input;
//   * 63-bit Morton codes (21 bits per axis) of every point in the root cube
//     of the paper's octree (Sec. 5.1) and a stable LSD radix sort of
//     (code, index) pairs -- points are stored along the Morton curve;
//   * a complete binary tree over buckets of kBucket consecutive points with
//     axis-aligned boxes, used by the exact k-nearest-neighbour search of
//     Eq. 7's face-to-point assignment;
//   * the octree of depth d around the cloud (Sec. 5.1, Alg. 1): every node
//     holding points is split into its 8 children down to depth d; empty
//     children are leaves of their own level.  Its leaves and their distinct
//     corners are the query points of the level-set step.
// All passes are HBM-bound scans, run once per cloud (or per depth change).
#include <algorithm>

#include "dwg_internal.cuh"

namespace dwg {

// ---------------------------------------------------------------------------
// input checks and bounding box
// ---------------------------------------------------------------------------
__global__ void k_check_finite(const float *__restrict__ v, int64_t cnt, int *err)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int bad = 0;
    for (; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(v[i])) bad = 1;
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(err, kErrNonfinite);
}

cudaError_t launch_check_finite(const float *v, int64_t cnt, int *err, cudaStream_t s)
{
    if (cnt <= 0) return cudaSuccess;
    unsigned blocks = (unsigned)std::min<int64_t>(ceil_div(cnt, 256), 4096);
    k_check_finite<<<blocks, 256, 0, s>>>(v, cnt, err);
    return cudaGetLastError();
}

__device__ __forceinline__ void atomic_min_f(float *a, float v)
{
    // order-preserving integer view of finite floats
    int iv = __float_as_int(v);
    if (iv >= 0) atomicMin((int *)a, iv);
    else atomicMax((unsigned *)a, (unsigned)iv);
}
__device__ __forceinline__ void atomic_max_f(float *a, float v)
{
    int iv = __float_as_int(v);
    if (iv >= 0) atomicMax((int *)a, iv);
    else atomicMin((unsigned *)a, (unsigned)iv);
}

__global__ void k_bbox_init(float *mm)
{
    if (threadIdx.x < 3) {
        mm[threadIdx.x] = INFINITY;
        mm[3 + threadIdx.x] = -INFINITY;
    }
}

__global__ void k_bbox(const float *__restrict__ xyz, int64_t n, float *mm)
{
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        for (int k = 0; k < 3; ++k) {
            float v = xyz[3 * i + k];
            lo[k] = fminf(lo[k], v);
            hi[k] = fmaxf(hi[k], v);
        }
    for (int k = 0; k < 3; ++k)
        for (int o = 16; o > 0; o >>= 1) {
            lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
            hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
        }
    if ((threadIdx.x & 31) == 0)
        for (int k = 0; k < 3; ++k) {
            atomic_min_f(&mm[k], lo[k]);
            atomic_max_f(&mm[3 + k], hi[k]);
        }
}

cudaError_t launch_bbox(const float *xyz, int64_t n, float *mm, cudaStream_t s)
{
    k_bbox_init<<<1, 32, 0, s>>>(mm);
    unsigned blocks = (unsigned)std::min<int64_t>(ceil_div(n, 256), 1024);
    k_bbox<<<blocks, 256, 0, s>>>(xyz, n, mm);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Morton codes
// ---------------------------------------------------------------------------
__global__ void k_morton(const float *__restrict__ xyz, int64_t n, double lo0, double lo1,
                         double lo2, double inv_h21, uint64_t *keys, int64_t *idx)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t cx = (uint64_t)quant21(xyz[3 * i + 0], lo0, inv_h21);
    uint64_t cy = (uint64_t)quant21(xyz[3 * i + 1], lo1, inv_h21);
    uint64_t cz = (uint64_t)quant21(xyz[3 * i + 2], lo2, inv_h21);
    keys[i] = morton3(cx, cy, cz);
    idx[i] = i;
}

cudaError_t launch_morton(const float *xyz, int64_t n, double lo0, double lo1, double lo2,
                          double inv_h21, uint64_t *keys, int64_t *idx, cudaStream_t s)
{
    k_morton<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(xyz, n, lo0, lo1, lo2, inv_h21, keys,
                                                         idx);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// exclusive scan of int64 (three phases: block sums, scan of sums, add)
// ---------------------------------------------------------------------------
constexpr int kScanBlock = 1024;
constexpr int kScanItems = 4;  // elements per thread

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t *sh, int64_t &total)
{
    // sh: blockDim.x int64 scratch
    int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int o = 1; o < blockDim.x; o <<= 1) {
        int64_t a = t >= o ? sh[t - o] : 0;
        __syncthreads();
        sh[t] += a;
        __syncthreads();
    }
    total = sh[blockDim.x - 1];
    int64_t incl = sh[t];
    __syncthreads();
    return incl - v;
}

__global__ void k_scan_block(const int64_t *__restrict__ in, int64_t *__restrict__ out, int64_t n,
                             int64_t *__restrict__ block_sums)
{
    __shared__ int64_t sh[kScanBlock];
    int64_t base = (int64_t)blockIdx.x * kScanBlock * kScanItems + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        v[k] = i < n ? in[i] : 0;
        s += v[k];
    }
    int64_t total;
    int64_t ex = block_exclusive_scan(s, sh, total);
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        if (i < n) out[i] = ex;
        ex += v[k];
    }
    if (threadIdx.x == 0 && block_sums) block_sums[blockIdx.x] = total;
}

__global__ void k_scan_add(int64_t *__restrict__ out, int64_t n, const int64_t *__restrict__ offs)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += offs[i / (kScanBlock * kScanItems)];
}

__global__ void k_scan_total(const int64_t *in, const int64_t *ex, int64_t n, int64_t *total)
{
    *total = n > 0 ? ex[n - 1] + in[n - 1] : 0;
}

// Exclusive scan of n int64 values; *d_total (device) receives the sum.
int scan_i64(Ctx *c, const int64_t *in, int64_t *out, int64_t n, int64_t *d_total)
{
    if (n <= 0) {
        DWG_CUDA_TRY(c, cudaMemsetAsync(d_total, 0, sizeof(int64_t), c->stream));
        return DWG_OK;
    }
    const int64_t per = (int64_t)kScanBlock * kScanItems;
    int64_t nb = ceil_div(n, per);
    if (nb == 1) {
        k_scan_block<<<1, kScanBlock, 0, c->stream>>>(in, out, n, nullptr);
    } else {
        int64_t *sums = nullptr, *soffs = nullptr, *stot = nullptr;
        DWG_CUDA_TRY(c, cudaMallocAsync(&sums, nb * sizeof(int64_t), c->stream));
        DWG_CUDA_TRY(c, cudaMallocAsync(&soffs, nb * sizeof(int64_t), c->stream));
        DWG_CUDA_TRY(c, cudaMallocAsync(&stot, sizeof(int64_t), c->stream));
        k_scan_block<<<(unsigned)nb, kScanBlock, 0, c->stream>>>(in, out, n, sums);
        int rc = scan_i64(c, sums, soffs, nb, stot);
        if (rc) return rc;
        k_scan_add<<<(unsigned)ceil_div(n, 256), 256, 0, c->stream>>>(out, n, soffs);
        cudaFreeAsync(sums, c->stream);
        cudaFreeAsync(soffs, c->stream);
        cudaFreeAsync(stot, c->stream);
    }
    k_scan_total<<<1, 1, 0, c->stream>>>(in, out, n, d_total);
    DWG_CUDA_TRY(c, cudaGetLastError());
    return DWG_OK;
}

// ---------------------------------------------------------------------------
// stable LSD radix sort of (uint64 key, int64 value) pairs, 8 bits per pass
// ---------------------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortItems = 8192;  // elements per block per pass

__global__ void k_sort_hist(const uint64_t *__restrict__ keys, int64_t n, int shift,
                            int64_t *__restrict__ hist, int nblocks)
{
    __shared__ unsigned h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t b0 = (int64_t)blockIdx.x * kSortItems;
    int64_t b1 = min(b0 + kSortItems, n);
    for (int64_t i = b0 + threadIdx.x; i < b1; i += kSortThreads)
        atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

__global__ void k_sort_scatter(const uint64_t *__restrict__ kin, const int64_t *__restrict__ vin,
                               int64_t n, int shift, const int64_t *__restrict__ offs,
                               int nblocks, uint64_t *__restrict__ kout,
                               int64_t *__restrict__ vout)
{
    constexpr int W = kSortThreads / 32;
    __shared__ unsigned cnt[W][256];
    __shared__ int64_t base[256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    base[threadIdx.x] = offs[(int64_t)threadIdx.x * nblocks + blockIdx.x];
    int64_t b0 = (int64_t)blockIdx.x * kSortItems;
    int64_t b1 = min(b0 + kSortItems, n);
    for (int64_t t0 = b0; t0 < b1; t0 += kSortThreads) {
        for (int w = 0; w < W; ++w) cnt[w][threadIdx.x] = 0;
        __syncthreads();
        int64_t i = t0 + threadIdx.x;
        bool valid = i < b1;
        uint64_t key = valid ? kin[i] : 0;
        unsigned dg = valid ? (unsigned)((key >> shift) & 255u) : 256u + lane;  // unique dummy
        unsigned peers = __match_any_sync(0xffffffffu, dg);
        unsigned rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && rank == 0) cnt[warp][dg] = __popc(peers);
        __syncthreads();
        // per digit: exclusive prefix over warps, running base
        {
            unsigned d = threadIdx.x;
            unsigned run = 0;
            for (int w = 0; w < W; ++w) {
                unsigned c = cnt[w][d];
                cnt[w][d] = run;
                run += c;
            }
            __syncthreads();
            if (valid) {
                int64_t dst = base[dg] + cnt[warp][dg] + rank;
                kout[dst] = key;
                vout[dst] = vin[i];
            }
            __syncthreads();
            base[d] += run;
        }
        __syncthreads();
    }
}

int radix_sort_pairs(Ctx *c, uint64_t *keys, int64_t *vals, int64_t n, int key_bits)
{
    if (n <= 1) return DWG_OK;
    int nblocks = (int)ceil_div(n, kSortItems);
    uint64_t *k2 = nullptr;
    int64_t *v2 = nullptr, *hist = nullptr, *offs = nullptr, *tot = nullptr;
    DWG_CUDA_TRY(c, cudaMallocAsync(&k2, n * sizeof(uint64_t), c->stream));
    DWG_CUDA_TRY(c, cudaMallocAsync(&v2, n * sizeof(int64_t), c->stream));
    DWG_CUDA_TRY(c, cudaMallocAsync(&hist, (int64_t)256 * nblocks * sizeof(int64_t), c->stream));
    DWG_CUDA_TRY(c, cudaMallocAsync(&offs, (int64_t)256 * nblocks * sizeof(int64_t), c->stream));
    DWG_CUDA_TRY(c, cudaMallocAsync(&tot, sizeof(int64_t), c->stream));
    uint64_t *ka = keys, *kb = k2;
    int64_t *va = vals, *vb = v2;
    int passes = (key_bits + 7) / 8;
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        k_sort_hist<<<nblocks, kSortThreads, 0, c->stream>>>(ka, n, shift, hist, nblocks);
        int rc = scan_i64(c, hist, offs, (int64_t)256 * nblocks, tot);
        if (rc) return rc;
        k_sort_scatter<<<nblocks, kSortThreads, 0, c->stream>>>(ka, va, n, shift, offs, nblocks,
                                                                  kb, vb);
        DWG_CUDA_TRY(c, cudaGetLastError());
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        DWG_CUDA_TRY(c, cudaMemcpyAsync(keys, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice,
                                        c->stream));
        DWG_CUDA_TRY(c, cudaMemcpyAsync(vals, va, n * sizeof(int64_t), cudaMemcpyDeviceToDevice,
                                        c->stream));
    }
    cudaFreeAsync(k2, c->stream);
    cudaFreeAsync(v2, c->stream);
    cudaFreeAsync(hist, c->stream);
    cudaFreeAsync(offs, c->stream);
    cudaFreeAsync(tot, c->stream);
    DWG_CUDA_TRY(c, cudaGetLastError());
    return DWG_OK;
}

// ---------------------------------------------------------------------------
// sorted points (x, y, z, a)
// ---------------------------------------------------------------------------
__global__ void k_gather_points(const float *__restrict__ xyz, const float *__restrict__ a,
                                const int64_t *__restrict__ perm, int64_t n, float4 *p4)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t j = perm[i];
    p4[i] = make_float4(xyz[3 * j], xyz[3 * j + 1], xyz[3 * j + 2], a ? a[j] : 1.f);
}

cudaError_t launch_gather_points(const float *xyz, const float *a, const int64_t *perm,
                                 int64_t n, float4 *p4, cudaStream_t s)
{
    k_gather_points<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(xyz, a, perm, n, p4);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// kNN bucket tree: heap-ordered complete binary tree, leaves = buckets
// ---------------------------------------------------------------------------
__global__ void k_bvh_leaves(const float4 *__restrict__ p4, int64_t n, int64_t nleaf,
                             float4 *lo, float4 *hi)
{
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nleaf) return;
    float4 l = make_float4(INFINITY, INFINITY, INFINITY, 0.f);
    float4 h = make_float4(-INFINITY, -INFINITY, -INFINITY, 0.f);
    int64_t j0 = b * kBucket, j1 = min(j0 + kBucket, n);
    for (int64_t j = j0; j < j1; ++j) {
        float4 p = p4[j];
        l.x = fminf(l.x, p.x); l.y = fminf(l.y, p.y); l.z = fminf(l.z, p.z);
        h.x = fmaxf(h.x, p.x); h.y = fmaxf(h.y, p.y); h.z = fmaxf(h.z, p.z);
    }
    lo[nleaf + b] = l;
    hi[nleaf + b] = h;
}

__global__ void k_bvh_level(int64_t first, int64_t count, float4 *lo, float4 *hi)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    int64_t nd = first + t;
    float4 a = lo[2 * nd], b = lo[2 * nd + 1], c = hi[2 * nd], d = hi[2 * nd + 1];
    lo[nd] = make_float4(fminf(a.x, b.x), fminf(a.y, b.y), fminf(a.z, b.z), 0.f);
    hi[nd] = make_float4(fmaxf(c.x, d.x), fmaxf(c.y, d.y), fmaxf(c.z, d.z), 0.f);
}

int build_knn_tree(Ctx *c)
{
    int64_t nb = ceil_div(c->n, kBucket);
    int L = 0;
    while (((int64_t)1 << L) < nb) ++L;
    c->knn_levels = L;
    int64_t nleaf = (int64_t)1 << L;
    DWG_CUDA_TRY(c, cudaMalloc(&c->d_bvh_lo, 2 * nleaf * sizeof(float4)));
    DWG_CUDA_TRY(c, cudaMalloc(&c->d_bvh_hi, 2 * nleaf * sizeof(float4)));
    k_bvh_leaves<<<(unsigned)ceil_div(nleaf, 256), 256, 0, c->stream>>>(c->d_p4, c->n, nleaf,
                                                                         c->d_bvh_lo, c->d_bvh_hi);
    for (int lv = L - 1; lv >= 0; --lv) {
        int64_t first = (int64_t)1 << lv;
        k_bvh_level<<<(unsigned)ceil_div(first, 256), 256, 0, c->stream>>>(first, first,
                                                                            c->d_bvh_lo,
                                                                            c->d_bvh_hi);
    }
    DWG_CUDA_TRY(c, cudaGetLastError());
    return DWG_OK;
}

// ---------------------------------------------------------------------------
// octree of depth d (Sec. 5.1): leaves and distinct corners
// ---------------------------------------------------------------------------
// flag[i] = 1 where the level-l prefix of code i starts a new node
__global__ void k_node_flags(const uint64_t *__restrict__ codes, int64_t n, int shift,
                             int64_t *flags)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    flags[i] = (i == 0 || (codes[i] >> shift) != (codes[i - 1] >> shift)) ? 1 : 0;
}

__global__ void k_node_compact(const uint64_t *__restrict__ codes, int64_t n, int shift,
                               const int64_t *__restrict__ flags, const int64_t *__restrict__ pos,
                               uint64_t *nodes)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !flags[i]) return;
    nodes[pos[i]] = codes[i] >> shift;
}

// child mask of each level-l node from the sorted level-(l+1) nodes
__global__ void k_child_mask(const uint64_t *__restrict__ parents, int64_t np,
                             const uint64_t *__restrict__ kids, int64_t nk, unsigned *mask)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nk) return;
    uint64_t pp = kids[i] >> 3;
    int64_t a = 0, b = np;
    while (a < b) {
        int64_t mid = (a + b) >> 1;
        if (parents[mid] < pp) a = mid + 1; else b = mid;
    }
    atomicOr(&mask[a], 1u << (unsigned)(kids[i] & 7));
}

__global__ void k_empty_count(const unsigned *__restrict__ mask, int64_t np, int64_t *cnt)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < np) cnt[i] = 8 - __popc(mask[i] & 255u);
}

// leaf record: x = level, y/z = prefix code (low/high 32 bits), w = nonempty
__global__ void k_emit_empty(const uint64_t *__restrict__ parents, int64_t np,
                             const unsigned *__restrict__ mask, const int64_t *__restrict__ pos,
                             int level_child, int64_t base, int4 *leaves)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    int64_t o = base + pos[i];
    unsigned mk = mask[i];
    for (int ch = 0; ch < 8; ++ch)
        if (!(mk & (1u << ch))) {
            uint64_t code = (parents[i] << 3) | (uint64_t)ch;
            leaves[o++] = make_int4(level_child, (int)(uint32_t)code, (int)(uint32_t)(code >> 32), 0);
        }
}

__global__ void k_emit_full(const uint64_t *__restrict__ nodes, int64_t nn, int level,
                            int64_t base, int4 *leaves)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    uint64_t code = nodes[i];
    leaves[base + i] = make_int4(level, (int)(uint32_t)code, (int)(uint32_t)(code >> 32), 1);
}

__device__ __forceinline__ void leaf_lattice(int4 L, int d, uint64_t &X, uint64_t &Y, uint64_t &Z,
                                             uint64_t &s)
{
    uint64_t code = (uint64_t)(uint32_t)L.y | ((uint64_t)(uint32_t)L.z << 32);
    s = 1ull << (d - L.x);
    X = compact3(code) * s;
    Y = compact3(code >> 1) * s;
    Z = compact3(code >> 2) * s;
}

// the 8 corners of every leaf as Morton keys of lattice points (value = slot)
__global__ void k_corner_keys(const int4 *__restrict__ leaves, int64_t nl, int d,
                              uint64_t *keys, int64_t *slots)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nl * 8) return;
    int64_t l = i >> 3;
    int v = (int)(i & 7);
    uint64_t X, Y, Z, s;
    leaf_lattice(leaves[l], d, X, Y, Z, s);
    keys[i] = morton3(X + (v & 1) * s, Y + ((v >> 1) & 1) * s, Z + ((v >> 2) & 1) * s);
    slots[i] = i;
}

__global__ void k_key_flags(const uint64_t *__restrict__ keys, int64_t m, int64_t *flags)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    flags[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

__global__ void k_corner_assign(const uint64_t *__restrict__ keys, const int64_t *__restrict__ slots,
                                const int64_t *__restrict__ flags, const int64_t *__restrict__ pos,
                                int64_t m, double lo0, double lo1, double lo2, double h,
                                int *leaf_corners, uint64_t *ukeys, float4 *upos)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    int64_t u = pos[i] + flags[i] - 1;  // index of this key's distinct corner
    leaf_corners[slots[i]] = (int)u;
    if (flags[i]) {
        uint64_t k = keys[i];
        double X = (double)compact3(k), Y = (double)compact3(k >> 1), Z = (double)compact3(k >> 2);
        ukeys[u] = k;
        upos[u] = make_float4((float)__dadd_rn(lo0, __dmul_rn(X, h)),
                              (float)__dadd_rn(lo1, __dmul_rn(Y, h)),
                              (float)__dadd_rn(lo2, __dmul_rn(Z, h)), 0.f);
    }
}

static void free_disc(Ctx *c)
{
    free_cell_lists(c);  // they index the leaves
    cudaFree(c->d_leaves);
    cudaFree(c->d_leaf_corners);
    cudaFree(c->d_corner_keys);
    cudaFree(c->d_corner_pos);
    cudaFree(c->d_wc);
    cudaFree(c->d_faces);
    cudaFree(c->d_defer);
    cudaFree(c->d_part_c);
    c->d_leaves = nullptr;
    c->d_leaf_corners = nullptr;
    c->d_corner_keys = nullptr;
    c->d_corner_pos = nullptr;
    c->d_wc = nullptr;
    c->d_faces = nullptr;
    c->d_defer = nullptr;
    c->d_part_c = nullptr;
    c->part_c_cap = 0;
    c->built_depth = -1;
}

static int read_count(Ctx *c, const int64_t *d_v, int64_t *h_v)
{
    DWG_CUDA_TRY(c, cudaMemcpyAsync(h_v, d_v, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
    DWG_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return DWG_OK;
}

int build_discretization(Ctx *c, int d)
{
    if (c->built_depth == d) return DWG_OK;
    free_disc(c);
    const int64_t n = c->n;
    const int B = 256;
    int64_t *flags = nullptr, *pos = nullptr, *tot = nullptr, *cnt = nullptr;
    uint64_t *nodes_a = nullptr, *nodes_b = nullptr;
    unsigned *mask = nullptr;
    int4 *leaves = nullptr;
    uint64_t *keys = nullptr;
    int64_t *slots = nullptr, *kf = nullptr, *kp = nullptr;

    auto body = [&]() -> int {
        DWG_CUDA_TRY(c, cudaMalloc(&flags, n * sizeof(int64_t)));
        DWG_CUDA_TRY(c, cudaMalloc(&pos, n * sizeof(int64_t)));
        DWG_CUDA_TRY(c, cudaMalloc(&cnt, n * sizeof(int64_t)));
        DWG_CUDA_TRY(c, cudaMalloc(&tot, sizeof(int64_t)));
        DWG_CUDA_TRY(c, cudaMalloc(&nodes_a, n * sizeof(uint64_t)));
        DWG_CUDA_TRY(c, cudaMalloc(&nodes_b, n * sizeof(uint64_t)));
        DWG_CUDA_TRY(c, cudaMalloc(&mask, n * sizeof(unsigned)));

        // unique level-l prefixes of the sorted codes, in Morton order
        auto level_nodes = [&](int lvl, uint64_t *out, int64_t &cntn) -> int {
            int shift = 3 * (kMortonBits - lvl);
            k_node_flags<<<(unsigned)ceil_div(n, B), B, 0, c->stream>>>(c->d_codes, n, shift,
                                                                         flags);
            int r = scan_i64(c, flags, pos, n, tot);
            if (r) return r;
            k_node_compact<<<(unsigned)ceil_div(n, B), B, 0, c->stream>>>(c->d_codes, n, shift,
                                                                           flags, pos, out);
            return read_count(c, tot, &cntn);
        };
        // pass 0 counts the leaves level by level, pass 1 emits them
        int64_t nleaves = 0;
        for (int pass = 0; pass < 2; ++pass) {
            int64_t base = 0, np = 0;
            int rc = level_nodes(0, nodes_a, np);
            if (rc) return rc;
            for (int lvl = 0; lvl < d; ++lvl) {
                int64_t nk = 0;
                if ((rc = level_nodes(lvl + 1, nodes_b, nk))) return rc;
                DWG_CUDA_TRY(c, cudaMemsetAsync(mask, 0, np * sizeof(unsigned), c->stream));
                k_child_mask<<<(unsigned)ceil_div(nk, B), B, 0, c->stream>>>(nodes_a, np, nodes_b,
                                                                              nk, mask);
                k_empty_count<<<(unsigned)ceil_div(np, B), B, 0, c->stream>>>(mask, np, cnt);
                if ((rc = scan_i64(c, cnt, pos, np, tot))) return rc;
                int64_t ne = 0;
                if ((rc = read_count(c, tot, &ne))) return rc;
                if (pass == 1 && ne > 0)
                    k_emit_empty<<<(unsigned)ceil_div(np, B), B, 0, c->stream>>>(
                        nodes_a, np, mask, pos, lvl + 1, base, leaves);
                base += ne;
                std::swap(nodes_a, nodes_b);
                np = nk;
            }
            if (pass == 1)  // non-empty leaves at depth d (nodes_a holds level d)
                k_emit_full<<<(unsigned)ceil_div(np, B), B, 0, c->stream>>>(nodes_a, np, d, base,
                                                                             leaves);
            base += np;
            if (pass == 0) {
                nleaves = base;
                DWG_CUDA_TRY(c, cudaMalloc(&leaves, nleaves * sizeof(int4)));
            }
        }
        DWG_CUDA_TRY(c, cudaGetLastError());

        // distinct corners: sort the 8 corner keys of every leaf, keep the first of each run
        int64_t m = nleaves * 8;
        DWG_CUDA_TRY(c, cudaMalloc(&keys, m * sizeof(uint64_t)));
        DWG_CUDA_TRY(c, cudaMalloc(&slots, m * sizeof(int64_t)));
        DWG_CUDA_TRY(c, cudaMalloc(&kf, m * sizeof(int64_t)));
        DWG_CUDA_TRY(c, cudaMalloc(&kp, m * sizeof(int64_t)));
        k_corner_keys<<<(unsigned)ceil_div(m, B), B, 0, c->stream>>>(leaves, nleaves, d, keys,
                                                                      slots);
        int rc = radix_sort_pairs(c, keys, slots, m, 3 * (d + 1));
        if (rc) return rc;
        k_key_flags<<<(unsigned)ceil_div(m, B), B, 0, c->stream>>>(keys, m, kf);
        if ((rc = scan_i64(c, kf, kp, m, tot))) return rc;
        int64_t nc = 0;
        if ((rc = read_count(c, tot, &nc))) return rc;
        DWG_CUDA_TRY(c, cudaMalloc(&c->d_leaf_corners, m * sizeof(int)));
        DWG_CUDA_TRY(c, cudaMalloc(&c->d_corner_keys, nc * sizeof(uint64_t)));
        DWG_CUDA_TRY(c, cudaMalloc(&c->d_corner_pos, nc * sizeof(float4)));
        double h = c->cube_L / (double)(1 << d);
        k_corner_assign<<<(unsigned)ceil_div(m, B), B, 0, c->stream>>>(
            keys, slots, kf, kp, m, c->cube_lo[0], c->cube_lo[1], c->cube_lo[2], h,
            c->d_leaf_corners, c->d_corner_keys, c->d_corner_pos);
        DWG_CUDA_TRY(c, cudaGetLastError());
        DWG_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        c->ncorners = nc;
        c->d_leaves = leaves;
        leaves = nullptr;
        c->nleaves = nleaves;
        c->max_faces = 6 * nleaves;
        DWG_CUDA_TRY(c, cudaMalloc(&c->d_wc, c->ncorners * sizeof(float)));
        DWG_CUDA_TRY(c, cudaMalloc(&c->d_faces, 2 * c->max_faces * sizeof(float4)));
        DWG_CUDA_TRY(c, cudaMalloc(&c->d_defer, kDeferCap * sizeof(int2)));
        // fixed-point scale of the face sums: 2^22 units per finest-cell area
        c->acc_scale = 4194304.0 / (h * h);
        c->built_depth = d;
        return DWG_OK;
    };
    int rc = body();
    cudaFree(keys);
    cudaFree(slots);
    cudaFree(kf);
    cudaFree(kp);
    cudaFree(leaves);
    cudaFree(flags);
    cudaFree(pos);
    cudaFree(cnt);
    cudaFree(tot);
    cudaFree(nodes_a);
    cudaFree(nodes_b);
    cudaFree(mask);
    if (rc) free_disc(c);
    return rc;
}

}  // namespace dwg
