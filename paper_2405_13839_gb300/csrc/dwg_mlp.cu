// dwg_mlp.cu -- the learned warm start: a kNN-patch MLP that proposes
// initial normals in place of the random ones of Sec. 5.1 (a project
// extension; the paper's options are random, PCA and Gauss-map normals).
//
// Network: 64 inputs (16 neighbour offsets scaled by the patch radius, the
// point's position relative to the cloud centroid, zero padding), three
// hidden layers of 64 with ReLU, 3 outputs (the normal before
// normalisation).  Weights and activations are rounded to bfloat16 and every
// layer is a tensor-core product with fp32 accumulation; biases, the loss
// and the optimiser state are fp32.
//
// Kernels:
//   k_mlp_forward_tc  rows of X -> Y (inference) on the tcgen05 tensor cores:
//                   128-row tiles, operands in shared memory, accumulators
//                   in tensor memory;
//   k_mlp_grad      forward + backward of the mean squared error over a
//                   batch on the warp-level tensor-core instruction
//                   (mma.sync m16n8k16, the fragments of one layer feed the
//                   next in registers): dY W4, dZ3 W3, dZ2 W2, weight
//                   gradients dZ^T H on tensor cores from per-warp shared
//                   stashes, summed per CTA in shared memory, then added to
//                   the global gradient;
//   k_adam          the Adam update of the fp32 master weights;
//   k_features      16 nearest neighbours (exact, the bucket-tree search)
//                   and the feature rows;
//   k_normals_from_y  normalise the network output into initial normals.
#include <cuda_bf16.h>

#include "dwg_internal.cuh"

namespace dwg {

constexpr int kOffW1 = 0, kOffB1 = 4096, kOffW2 = 4160, kOffB2 = 8256, kOffW3 = 8320,
              kOffB3 = 12416, kOffW4 = 12480, kOffB4 = 12672;
constexpr int kMlpParams = 12675;
constexpr int kMlpWarps = 4;           // 16 rows per warp, 64 rows per CTA
constexpr int kMlpRows = 16 * kMlpWarps;

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}
__device__ __forceinline__ uint16_t bf16_bits(float x)
{
    __nv_bfloat16 v = __float2bfloat16_rn(x);
    return *reinterpret_cast<uint16_t *>(&v);
}
__device__ __forceinline__ uint32_t pair16(uint16_t lo, uint16_t hi)
{
    return (uint32_t)lo | ((uint32_t)hi << 16);
}

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// shared-memory copy of the weights (bf16) and biases (fp32)
struct MlpSmem {
    uint16_t W[3][64 * 64];   // W1, W2, W3 as [out][in]
    uint16_t W4[8 * 64];      // W4 padded to 8 outputs
    float b[3][64];
    float b4[8];
};
struct MlpSmemT {
    uint16_t Wt[2][64 * 64];  // W2^T, W3^T as [in][out]
    uint16_t W4t[64 * 16];    // W4^T padded to 16 columns
};

__device__ void load_weights(const float *__restrict__ P, MlpSmem &S, MlpSmemT *T)
{
    for (int i = threadIdx.x; i < 64 * 64; i += blockDim.x) {
        S.W[0][i] = bf16_bits(P[kOffW1 + i]);
        S.W[1][i] = bf16_bits(P[kOffW2 + i]);
        S.W[2][i] = bf16_bits(P[kOffW3 + i]);
        if (T) {
            int o = i / 64, in = i % 64;  // W[o][in] -> Wt[in][o]
            T->Wt[0][in * 64 + o] = S.W[1][i];
            T->Wt[1][in * 64 + o] = S.W[2][i];
        }
    }
    for (int i = threadIdx.x; i < 8 * 64; i += blockDim.x)
        S.W4[i] = i < 3 * 64 ? bf16_bits(P[kOffW4 + i]) : (uint16_t)0;
    if (T)
        for (int i = threadIdx.x; i < 64 * 16; i += blockDim.x) {
            int f = i / 16, c = i % 16;
            T->W4t[i] = c < 3 ? bf16_bits(P[kOffW4 + c * 64 + f]) : (uint16_t)0;
        }
    for (int i = threadIdx.x; i < 64; i += blockDim.x) {
        S.b[0][i] = P[kOffB1 + i];
        S.b[1][i] = P[kOffB2 + i];
        S.b[2][i] = P[kOffB3 + i];
    }
    if (threadIdx.x < 8) S.b4[threadIdx.x] = threadIdx.x < 3 ? P[kOffB4 + threadIdx.x] : 0.f;
}

// A fragments of 16 rows of X (fp32, row-major, 64 columns) -> bf16
__device__ __forceinline__ void load_x(const float *__restrict__ X, int64_t row0, int64_t B,
                                       uint32_t (&a)[4][4], int lane)
{
    const int g = lane >> 2, t = lane & 3;
    const int64_t r0 = row0 + g, r1 = row0 + g + 8;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        float2 v00 = r0 < B ? *reinterpret_cast<const float2 *>(X + r0 * 64 + 16 * kk + 2 * t)
                            : make_float2(0.f, 0.f);
        float2 v10 = r1 < B ? *reinterpret_cast<const float2 *>(X + r1 * 64 + 16 * kk + 2 * t)
                            : make_float2(0.f, 0.f);
        float2 v01 = r0 < B ? *reinterpret_cast<const float2 *>(X + r0 * 64 + 16 * kk + 8 + 2 * t)
                            : make_float2(0.f, 0.f);
        float2 v11 = r1 < B ? *reinterpret_cast<const float2 *>(X + r1 * 64 + 16 * kk + 8 + 2 * t)
                            : make_float2(0.f, 0.f);
        a[kk][0] = pack_bf16(v00.x, v00.y);
        a[kk][1] = pack_bf16(v10.x, v10.y);
        a[kk][2] = pack_bf16(v01.x, v01.y);
        a[kk][3] = pack_bf16(v11.x, v11.y);
    }
}

// acc[nt] = A (16 x 64) x W^T for the 8 output tiles of one layer
__device__ __forceinline__ void layer_mma(const uint16_t *__restrict__ W, const uint32_t (&a)[4][4],
                                          float (&acc)[8][4], int lane)
{
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const uint16_t *row = W + (8 * nt + g) * 64 + 16 * kk + 2 * t;
            mma16816(acc[nt], a[kk], *reinterpret_cast<const uint32_t *>(row),
                     *reinterpret_cast<const uint32_t *>(row + 8));
        }
}

// bias + ReLU, the relu mask (bit nt*4+e), and the next layer's A fragments
__device__ __forceinline__ void bias_relu(float (&acc)[8][4], const float *__restrict__ b,
                                          uint32_t (&a)[4][4], uint32_t &mask, int lane)
{
    const int t = lane & 3;
    mask = 0;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            float z = acc[nt][e] + b[8 * nt + 2 * t + (e & 1)];
            if (z > 0.f) mask |= 1u << (nt * 4 + e);
            acc[nt][e] = z > 0.f ? z : 0.f;
        }
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        a[kk][0] = pack_bf16(acc[2 * kk][0], acc[2 * kk][1]);
        a[kk][1] = pack_bf16(acc[2 * kk][2], acc[2 * kk][3]);
        a[kk][2] = pack_bf16(acc[2 * kk + 1][0], acc[2 * kk + 1][1]);
        a[kk][3] = pack_bf16(acc[2 * kk + 1][2], acc[2 * kk + 1][3]);
    }
}

// the output layer: y (16 x 8, first 3 columns used)
__device__ __forceinline__ void out_layer(const MlpSmem &S, const uint32_t (&a)[4][4],
                                          float (&y)[4], int lane)
{
    const int g = lane >> 2, t = lane & 3;
    y[0] = y[1] = y[2] = y[3] = 0.f;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const uint16_t *row = S.W4 + g * 64 + 16 * kk + 2 * t;
        mma16816(y, a[kk], *reinterpret_cast<const uint32_t *>(row),
                 *reinterpret_cast<const uint32_t *>(row + 8));
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) y[e] += S.b4[2 * t + (e & 1)];
}

// --- inference on the 5th-generation tensor cores (tcgen05) -----------------
//
// One CTA of 128 threads runs tiles of 128 rows (persistent over the tiles).
// Every layer is D (128 x N, fp32, in tensor memory) = A (128 x 64, bf16,
// shared memory) x W^T (W: N x 64 bf16, shared memory), issued by one thread
// as four K = 16 steps of tcgen05.mma (kind::f16, M = 128, N = 64, or 16 for
// the output layer whose rows 3..15 are zero).  Both operands are K-major
// in the canonical no-swizzle layout: 8 x 16-byte core matrices, 128 bytes
// apart along K (leading byte offset) and 1024 bytes apart along the rows
// (stride byte offset).  tcgen05.commit signals an mbarrier when the layer's
// MMAs are done; each thread then reads its row (thread t = tensor-memory
// lane t) with tcgen05.ld, adds the bias, applies ReLU, rounds to bf16 and
// writes the row back into the A buffer for the next layer.
constexpr int kTcRows = 128;
constexpr int kTcCols = 64;  // tensor-memory columns (fp32 accumulator of N <= 64)

struct MlpTcSmem {
    uint16_t W[3][64 * 64];   // canonical K-major layout, see tc_off
    uint16_t W4[16 * 64];     // output layer, rows 3..15 zero
    uint16_t A[kTcRows * 64]; // activations of the current layer
    float b[3][64];
    float b4[16];
    uint64_t bar;
    uint32_t tmem_base;
};

// element (r, k) of a K-major bf16 operand with 64 columns: core matrix
// (r / 8, k / 8) of 8 rows x 16 bytes, cores 128 bytes apart along K
__device__ __forceinline__ int tc_off(int r, int k)
{
    return (((r >> 3) * 8 + (k >> 3)) * 64) + (r & 7) * 8 + (k & 7);  // in bf16 elements
}

// shared-memory matrix descriptor: start address, leading byte offset 128,
// stride byte offset 1024, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t tc_desc(const void *p)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    uint64_t d = (uint64_t)((a & 0x3FFFFu) >> 4);
    d |= (uint64_t)(128u >> 4) << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor, kind::f16: fp32 accumulator, bf16 A and B, both
// K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t tc_idesc(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(kTcRows >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                       uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t *bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            (uint32_t)__cvta_generic_to_shared(bar))
        : "memory");
}

__device__ __forceinline__ bool tc_wait(uint64_t *bar, uint32_t parity)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(bar);
    for (int it = 0; it < (1 << 24); ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// 16 consecutive fp32 columns of this thread's lane
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(kTcRows)
    k_mlp_forward_tc(const float *__restrict__ P, const float *__restrict__ X, int64_t B,
                     float *__restrict__ Y, int *__restrict__ err)
{
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    MlpTcSmem &S = *reinterpret_cast<MlpTcSmem *>(tc_smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5;
    // weights and biases, bf16 in the canonical layout
    for (int i = tid; i < 64 * 64; i += kTcRows) {
        const int o = i / 64, k = i % 64;
        S.W[0][tc_off(o, k)] = bf16_bits(P[kOffW1 + i]);
        S.W[1][tc_off(o, k)] = bf16_bits(P[kOffW2 + i]);
        S.W[2][tc_off(o, k)] = bf16_bits(P[kOffW3 + i]);
    }
    for (int i = tid; i < 16 * 64; i += kTcRows) {
        const int o = i / 64, k = i % 64;
        S.W4[tc_off(o, k)] = o < 3 ? bf16_bits(P[kOffW4 + i]) : (uint16_t)0;
    }
    for (int i = tid; i < 64; i += kTcRows) {
        S.b[0][i] = P[kOffB1 + i];
        S.b[1][i] = P[kOffB2 + i];
        S.b[2][i] = P[kOffB3 + i];
    }
    if (tid < 16) S.b4[tid] = tid < 3 ? P[kOffB4 + tid] : 0.f;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(&S.bar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(&S.tmem_base)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = S.tmem_base;
    const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);  // this warp's lanes
    uint32_t phase = 0;
    bool ok = true;
    const int64_t ntiles = (B + kTcRows - 1) / kTcRows;
    // a tile's rows of X, coalesced float4 reads (element e = tid + 128 i is
    // row e / 16, columns 4 (e % 16) ..); the next tile's are loaded while
    // the current tile's layers run
    float4 xr[16];
    auto load_x = [&](int64_t t) {
        const int64_t r0 = t * kTcRows;
        const float4 *X4 = reinterpret_cast<const float4 *>(X + r0 * 64);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int e = tid + kTcRows * i;
            xr[i] = r0 + (e >> 4) < B ? X4[e] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    if ((int64_t)blockIdx.x < ntiles) load_x(blockIdx.x);
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int64_t row0 = tile * kTcRows;
#pragma unroll
        for (int i = 0; i < 16; ++i) {  // -> bf16 A
            const int e = tid + kTcRows * i, r = e >> 4, c4 = e & 15;
            *reinterpret_cast<uint2 *>(&S.A[tc_off(r, 4 * c4)]) =
                make_uint2(pack_bf16(xr[i].x, xr[i].y), pack_bf16(xr[i].z, xr[i].w));
        }
        if (tile + gridDim.x < ntiles) load_x(tile + gridDim.x);
        for (int l = 0; l < 4 && ok; ++l) {
            const uint16_t *W = l < 3 ? S.W[l] : S.W4;
            const int N = l < 3 ? 64 : 16;
            // A written by the threads -> visible to the tensor cores
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t idesc = tc_idesc(N);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    tc_mma(tmem, tc_desc(&S.A[tc_off(0, 16 * kk)]), tc_desc(&W[tc_off(0, 16 * kk)]),
                           idesc, kk > 0 ? 1u : 0u);
                tc_commit(&S.bar);
            }
            // every thread waits; the outcome is made uniform before anyone
            // leaves the loop, so that no barrier below is skipped by a part
            // of the block
            const bool got = tc_wait(&S.bar, phase);
            if (!__syncthreads_and(got)) {
                ok = false;
                if (tid == 0) atomicOr(err, kErrTimeout);
                break;
            }
            phase ^= 1u;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int r = tid;
            if (l < 3) {
                const float *bias = S.b[l];
#pragma unroll
                for (int c0 = 0; c0 < 64; c0 += 16) {
                    float v[16];
                    tc_ld16(lane_addr + (uint32_t)c0, v);
#pragma unroll
                    for (int i = 0; i < 16; i += 4) {
                        float z0 = fmaxf(v[i] + bias[c0 + i], 0.f);
                        float z1 = fmaxf(v[i + 1] + bias[c0 + i + 1], 0.f);
                        float z2 = fmaxf(v[i + 2] + bias[c0 + i + 2], 0.f);
                        float z3 = fmaxf(v[i + 3] + bias[c0 + i + 3], 0.f);
                        *reinterpret_cast<uint2 *>(&S.A[tc_off(r, c0 + i)]) =
                            make_uint2(pack_bf16(z0, z1), pack_bf16(z2, z3));
                    }
                }
            } else {
                float v[16];
                tc_ld16(lane_addr, v);
                if (row0 + r < B) {
                    Y[(row0 + r) * 3 + 0] = v[0] + S.b4[0];
                    Y[(row0 + r) * 3 + 1] = v[1] + S.b4[1];
                    Y[(row0 + r) * 3 + 2] = v[2] + S.b4[2];
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();  // A and the accumulator are reused by the next tile
    }
    if (!ok && tid == 0) {
        // let any MMA still in flight finish (bounded) before the memory goes
        tc_wait(&S.bar, phase);
    }
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTcCols)
                     : "memory");
}

// --- training -------------------------------------------------------------
struct MlpGradSmem {
    float gW[3][64 * 64];
    float gW4[3 * 64];
    float gb[3][64];
    float gb4[4];
};
struct MlpStash {
    uint16_t act[4][16 * 64];  // x, h1, h2, h3 of the warp's 16 rows, bf16
    uint16_t dz[16 * 64];      // the current layer's dZ, bf16
    uint16_t dy[16 * 16];      // dY padded to 16 columns
};

// store a C-layout tile set (16 x 64) as bf16 rows in a stash
__device__ __forceinline__ void stash_c(const float (&v)[8][4], uint16_t *dst, int lane)
{
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        int c = 8 * nt + 2 * t;
        *reinterpret_cast<uint32_t *>(dst + g * 64 + c) = pack_bf16(v[nt][0], v[nt][1]);
        *reinterpret_cast<uint32_t *>(dst + (g + 8) * 64 + c) = pack_bf16(v[nt][2], v[nt][3]);
    }
}
__device__ __forceinline__ void stash_a(const uint32_t (&a)[4][4], uint16_t *dst, int lane)
{
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        *reinterpret_cast<uint32_t *>(dst + g * 64 + 16 * kk + 2 * t) = a[kk][0];
        *reinterpret_cast<uint32_t *>(dst + (g + 8) * 64 + 16 * kk + 2 * t) = a[kk][1];
        *reinterpret_cast<uint32_t *>(dst + g * 64 + 16 * kk + 8 + 2 * t) = a[kk][2];
        *reinterpret_cast<uint32_t *>(dst + (g + 8) * 64 + 16 * kk + 8 + 2 * t) = a[kk][3];
    }
}

// gW[o][f] += sum_s D[s][o] * H[s][f] over the warp's 16 rows (tensor cores);
// D is (16 x ncols_d) bf16 with row stride ld_d, H is (16 x 64) bf16
__device__ __forceinline__ void weight_grad(const uint16_t *D, int ld_d, int mtiles,
                                            const uint16_t *H, float *gW, int rows_out, int lane)
{
    const int g = lane >> 2, t = lane & 3;
    for (int mt = 0; mt < mtiles; ++mt) {
        uint32_t a[4];
        int o0 = 16 * mt + g, o1 = o0 + 8;
        a[0] = pair16(D[(2 * t) * ld_d + o0], D[(2 * t + 1) * ld_d + o0]);
        a[1] = pair16(D[(2 * t) * ld_d + o1], D[(2 * t + 1) * ld_d + o1]);
        a[2] = pair16(D[(2 * t + 8) * ld_d + o0], D[(2 * t + 9) * ld_d + o0]);
        a[3] = pair16(D[(2 * t + 8) * ld_d + o1], D[(2 * t + 9) * ld_d + o1]);
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            int f = 8 * nt + g;
            uint32_t b0 = pair16(H[(2 * t) * 64 + f], H[(2 * t + 1) * 64 + f]);
            uint32_t b1 = pair16(H[(2 * t + 8) * 64 + f], H[(2 * t + 9) * 64 + f]);
            float d[4] = {0.f, 0.f, 0.f, 0.f};
            mma16816(d, a, b0, b1);
            int c = 8 * nt + 2 * t;
            if (o0 < rows_out) {
                atomicAdd(&gW[o0 * 64 + c], d[0]);
                atomicAdd(&gW[o0 * 64 + c + 1], d[1]);
            }
            if (o1 < rows_out) {
                atomicAdd(&gW[o1 * 64 + c], d[2]);
                atomicAdd(&gW[o1 * 64 + c + 1], d[3]);
            }
        }
    }
}

// column sums of a C-layout tile set over the warp's 16 rows -> gb
__device__ __forceinline__ void bias_grad(const float (&v)[8][4], float *gb, int lane)
{
    const int t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            float s = v[nt][e] + v[nt][e + 2];
            s += __shfl_xor_sync(0xffffffffu, s, 4);
            s += __shfl_xor_sync(0xffffffffu, s, 8);
            s += __shfl_xor_sync(0xffffffffu, s, 16);
            if (lane < 4) atomicAdd(&gb[8 * nt + 2 * t + e], s);
        }
}

// dH (16 x 64) = dZ (16 x 64, as A fragments) x W (B operand [in][out] = W^T rows)
__device__ __forceinline__ void back_mma(const uint16_t *Wt, const uint32_t (&a)[4][4],
                                         float (&acc)[8][4], int lane)
{
    layer_mma(Wt, a, acc, lane);
}

__global__ void __launch_bounds__(32 * kMlpWarps)
    k_mlp_grad(const float *__restrict__ P, const float *__restrict__ X,
               const float *__restrict__ T, int64_t B, float *__restrict__ grad,
               double *__restrict__ loss)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MlpSmem &S = *reinterpret_cast<MlpSmem *>(smem_raw);
    MlpSmemT &ST = *reinterpret_cast<MlpSmemT *>(smem_raw + sizeof(MlpSmem));
    MlpGradSmem &G =
        *reinterpret_cast<MlpGradSmem *>(smem_raw + sizeof(MlpSmem) + sizeof(MlpSmemT));
    MlpStash *stash = reinterpret_cast<MlpStash *>(smem_raw + sizeof(MlpSmem) + sizeof(MlpSmemT) +
                                                   sizeof(MlpGradSmem));
    load_weights(P, S, &ST);
    {
        float *z = reinterpret_cast<float *>(&G);
        for (int i = threadIdx.x; i < (int)(sizeof(MlpGradSmem) / sizeof(float)); i += blockDim.x)
            z[i] = 0.f;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    MlpStash &W = stash[warp];
    const float inv2b = 2.f / (float)B;
    double lsum = 0.0;
    for (int64_t row0 = ((int64_t)blockIdx.x * kMlpWarps + warp) * 16; row0 < B;
         row0 += (int64_t)gridDim.x * kMlpRows) {
        uint32_t a[4][4], mask[3];
        float acc[8][4], y[4];
        load_x(X, row0, B, a, lane);
        stash_a(a, W.act[0], lane);
        for (int l = 0; l < 3; ++l) {
            layer_mma(S.W[l], a, acc, lane);
            bias_relu(acc, S.b[l], a, mask[l], lane);
            stash_a(a, W.act[l + 1], lane);
        }
        out_layer(S, a, y, lane);
        // dY = 2 (y - t) / B for the valid rows and the 3 used columns
        float dyv[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            int col = 2 * t + (e & 1);
            int64_t r = row0 + g + (e >= 2 ? 8 : 0);
            float d = 0.f;
            if (col < 3 && r < B) {
                float res = y[e] - T[r * 3 + col];
                lsum += (double)res * (double)res;
                d = res * inv2b;
            }
            dyv[e] = d;
        }
        __syncwarp();
        // stash dY (16 x 16) and take its A fragment (columns 0..7 carry data)
        *reinterpret_cast<uint32_t *>(W.dy + g * 16 + 2 * t) = pack_bf16(dyv[0], dyv[1]);
        *reinterpret_cast<uint32_t *>(W.dy + (g + 8) * 16 + 2 * t) = pack_bf16(dyv[2], dyv[3]);
        *reinterpret_cast<uint32_t *>(W.dy + g * 16 + 8 + 2 * t) = 0u;
        *reinterpret_cast<uint32_t *>(W.dy + (g + 8) * 16 + 8 + 2 * t) = 0u;
        uint32_t ad[4][4];
        ad[0][0] = pack_bf16(dyv[0], dyv[1]);
        ad[0][1] = pack_bf16(dyv[2], dyv[3]);
        ad[0][2] = 0u;
        ad[0][3] = 0u;
        // db4 (columns 0..2)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            float s = dyv[e] + dyv[e + 2];
            s += __shfl_xor_sync(0xffffffffu, s, 4);
            s += __shfl_xor_sync(0xffffffffu, s, 8);
            s += __shfl_xor_sync(0xffffffffu, s, 16);
            if (lane < 4 && 2 * t + e < 3) atomicAdd(&G.gb4[2 * t + e], s);
        }
        __syncwarp();
        // dW4 (3 x 64) = dY^T h3
        weight_grad(W.dy, 16, 1, W.act[3], G.gW4, 3, lane);
        // dH3 = dY W4 (K = 16, dY columns 3..15 are zero)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
            const uint16_t *row = ST.W4t + (8 * nt + g) * 16 + 2 * t;
            mma16816(acc[nt], ad[0], *reinterpret_cast<const uint32_t *>(row),
                     *reinterpret_cast<const uint32_t *>(row + 8));
        }
        // layers 3, 2, 1: dZ = dH * relu'(Z); db, dW; dH_prev = dZ W
        for (int l = 2; l >= 0; --l) {
#pragma unroll
            for (int nt = 0; nt < 8; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (!(mask[l] & (1u << (nt * 4 + e)))) acc[nt][e] = 0.f;
            bias_grad(acc, G.gb[l], lane);
            __syncwarp();
            stash_c(acc, W.dz, lane);
            __syncwarp();
            weight_grad(W.dz, 64, 4, W.act[l], G.gW[l], 64, lane);
            if (l > 0) {
                uint32_t az[4][4];
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    az[kk][0] = pack_bf16(acc[2 * kk][0], acc[2 * kk][1]);
                    az[kk][1] = pack_bf16(acc[2 * kk][2], acc[2 * kk][3]);
                    az[kk][2] = pack_bf16(acc[2 * kk + 1][0], acc[2 * kk + 1][1]);
                    az[kk][3] = pack_bf16(acc[2 * kk + 1][2], acc[2 * kk + 1][3]);
                }
                back_mma(ST.Wt[l - 1], az, acc, lane);
            }
            __syncwarp();
        }
    }
    // loss and the CTA's gradient sums
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (lane == 0) atomicAdd(loss, lsum / (double)B);
    __syncthreads();
    for (int i = threadIdx.x; i < 64 * 64; i += blockDim.x) {
        atomicAdd(&grad[kOffW1 + i], G.gW[0][i]);
        atomicAdd(&grad[kOffW2 + i], G.gW[1][i]);
        atomicAdd(&grad[kOffW3 + i], G.gW[2][i]);
    }
    for (int i = threadIdx.x; i < 64; i += blockDim.x) {
        atomicAdd(&grad[kOffB1 + i], G.gb[0][i]);
        atomicAdd(&grad[kOffB2 + i], G.gb[1][i]);
        atomicAdd(&grad[kOffB3 + i], G.gb[2][i]);
    }
    for (int i = threadIdx.x; i < 3 * 64; i += blockDim.x) atomicAdd(&grad[kOffW4 + i], G.gW4[i]);
    if (threadIdx.x < 3) atomicAdd(&grad[kOffB4 + threadIdx.x], G.gb4[threadIdx.x]);
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, int n, float lr, float b1, float b2, float eps,
                       float bc1, float bc2)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float gi = g[i];
    float mi = b1 * m[i] + (1.f - b1) * gi;
    float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

size_t mlp_grad_smem_bytes()
{
    return sizeof(MlpSmem) + sizeof(MlpSmemT) + sizeof(MlpGradSmem) + kMlpWarps * sizeof(MlpStash);
}

static int mlp_sms()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 148;
}

// device flag for the forward calls that have no handle (dwg_mlp_forward)
static __device__ int g_mlp_err;

cudaError_t launch_mlp_forward(const float *P, const float *X, int64_t B, float *Y, cudaStream_t s,
                               int *err)
{
    if (!err) {
        cudaError_t e = cudaGetSymbolAddress((void **)&err, g_mlp_err);
        if (e != cudaSuccess) return e;
    }
    int64_t blocks = std::min<int64_t>(ceil_div(B, kTcRows), (int64_t)mlp_sms() * 4);
    k_mlp_forward_tc<<<(unsigned)std::max<int64_t>(blocks, 1), kTcRows, sizeof(MlpTcSmem), s>>>(
        P, X, B, Y, err);
    return cudaGetLastError();
}

int mlp_forward_error(cudaStream_t s)
{
    int *d = nullptr, h = 0;
    if (cudaGetSymbolAddress((void **)&d, g_mlp_err) != cudaSuccess) return -1;
    if (cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return -1;
    if (h) cudaMemsetAsync(d, 0, sizeof(int), s);
    return h;
}

cudaError_t launch_mlp_grad(const float *P, const float *X, const float *T, int64_t B, float *grad,
                            double *loss, cudaStream_t s)
{
    size_t sm = mlp_grad_smem_bytes();
    cudaError_t e =
        cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(grad, 0, kMlpParams * sizeof(float), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(loss, 0, sizeof(double), s)) != cudaSuccess) return e;
    int64_t blocks = std::min<int64_t>(ceil_div(B, kMlpRows), (int64_t)mlp_sms());
    k_mlp_grad<<<(unsigned)std::max<int64_t>(blocks, 1), 32 * kMlpWarps, sm, s>>>(P, X, T, B, grad,
                                                                               loss);
    return cudaGetLastError();
}

cudaError_t launch_adam(float *p, const float *g, float *m, float *v, int step, float lr,
                        cudaStream_t s)
{
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    float bc1 = 1.f - powf(b1, (float)step), bc2 = 1.f - powf(b2, (float)step);
    k_adam<<<(unsigned)ceil_div(kMlpParams, 256), 256, 0, s>>>(p, g, m, v, kMlpParams, lr, b1, b2,
                                                               eps, bc1, bc2);
    return cudaGetLastError();
}

}  // namespace dwg
