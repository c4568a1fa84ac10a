// dwg_eval.cu -- exact all-pairs evaluation of the generalized winding
// number and its gradient (paper Sec. 3, Eq. 2/3; screened variant Sec. 4.2,
// Eq. 5) on sm_103a.
//
// Work decomposition: a CTA of NT threads (128 or 256) owns a tile of
// NT * 2P queries (each thread holds P query pairs in registers) and one
// contiguous chunk of the sources; (P, NT) is a tuning choice (one
// instantiation per shape, picked at run time).  Source records (48 bytes: x, y, z, mx, my, mz, each stored
// twice so that one 64-bit register pair feeds both lanes of a packed
// f32x2 instruction) stream through a 4-stage shared-memory ring filled by
// the bulk-copy (TMA) engine with mbarrier completion.  Every thread reads
// each record by broadcast and updates its 2P queries with packed
// fma/mul/add.f32x2 instructions; rsqrt (and ex2 for the screened kernel)
// run on the MUFU unit.
//
// Precision: terms are FP32.  Each thread sums one 128-source tile in plain
// FP32 and folds the tile sum into a (hi, lo) two-sum pair, so the long sum
// over all sources is compensated.  The CTA writes its (hi, lo) partials for
// its source chunk; a reduce kernel combines the chunks in a fixed order
// (deterministic) and adds back the exactly-known coincident-point terms.
//
// Per term, with d = p - q, rho^2 = |d|^2 + eps^2, m = a n / (4 pi),
// inv = rho^-1:
//   plain    w += <m,d> inv^3;   grad += 3 <m,d> inv^5 d - m inv^3
//   screened F = exp(-s rho)(1 + s rho):
//            w += F <m,d> inv^3;
//            grad += <m,d> inv^3 (3 F inv^2 + s^2 exp(-s rho)) d - F inv^3 m
// A source equal to the query (d = 0) contributes exactly zero to w and to
// the d-terms; its only contribution, -F inv^3 m to the gradient, is
// subtracted after the sum (reduce kernel), which skips it exactly as the
// definition requires without a per-term test.
#include "dwg_internal.cuh"
#include "dwg_packed.cuh"

namespace dwg {

// ---------------------------------------------------------------------------
// mbarrier + bulk copy (inline PTX), with bounded waits
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Returns false when the wait gave up (by default about 2^24 polls, well
// beyond any copy latency); the caller then reports DWG_ERR_TIMEOUT.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  int limit = 1 << 24)
{
    for (int it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Self-check of the wait limit: an mbarrier that expects one arrival which
// never comes (no copy is issued), waited on with `polls` polls through the
// evaluators' bounded wait; the timeout is recorded like a stalled copy's.
__global__ void k_wait_selfcheck(int polls, int *err)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, 0, polls)) atomicOr(err, kErrTimeout);
    __syncthreads();
}

cudaError_t launch_wait_selfcheck(Ctx *c, int polls)
{
    k_wait_selfcheck<<<1, 32, 0, c->stream>>>(polls, c->d_err);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP32 issue microbenchmarks (the denominators of the evaluators' roofline)
// ---------------------------------------------------------------------------
// Packed FMA: each thread runs 8 independent chains of fma.rn.f32x2, `iters`
// times; one packed instruction is 2 FP32 lane operations.  The chains
// converge to a fixed point, so no value overflows; the result is written
// only under a condition that never holds, which keeps the work.
__global__ void __launch_bounds__(256) k_peak_ffma(int iters, float seed, float *sink)
{
    f2 x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = pk(seed + k + threadIdx.x * 1e-3f, seed - k);
    const f2 a = pk(0.5f, 0.5f), b = pk(0.25f, 0.25f);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma2(x[k], a, b);
    }
    float s0 = 0.f, s1 = 0.f, lo, hi;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        upk(x[k], lo, hi);
        s0 += lo;
        s1 += hi;
    }
    if (s0 + s1 == -1.f) sink[blockIdx.x] = s0;
}

// MUFU reciprocal square root: 8 independent chains y <- rsqrt(y) (a fixed
// point at 1), `iters` times.
__global__ void __launch_bounds__(256) k_peak_rsqrt(int iters, float seed, float *sink)
{
    float y[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) y[k] = seed + 0.1f * k + threadIdx.x * 1e-4f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) y[k] = rsqrt_mufu(y[k]);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += y[k];
    if (s == -1.f) sink[blockIdx.x] = s;
}

// MUFU base-2 exponential: 8 independent chains y <- 2^(-y) (a fixed point
// near 0.641), `iters` times.
__global__ void __launch_bounds__(256) k_peak_ex2(int iters, float seed, float *sink)
{
    float y[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) y[k] = seed + 0.01f * k + threadIdx.x * 1e-5f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) y[k] = ex2_mufu(-y[k]);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += y[k];
    if (s == -1.f) sink[blockIdx.x] = s;
}

int measure_fp32_peaks(int device, double *ffma_lane_ops, double *rsqrt_ops, double *ex2_ops)
{
    cudaSetDevice(device);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (sms < 1) return DWG_ERR_CUDA;
    const int blocks = sms * 8, threads = 256;
    float *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = DWG_OK;
    auto timed = [&](int which, int iters, double *ms) -> bool {
        cudaEventRecord(e0);
        if (which == 0) k_peak_ffma<<<blocks, threads>>>(iters, 1.0f, sink);
        else if (which == 1) k_peak_rsqrt<<<blocks, threads>>>(iters, 1.5f, sink);
        else k_peak_ex2<<<blocks, threads>>>(iters, 0.6f, sink);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess) return false;
        float f = 0.f;
        cudaEventElapsedTime(&f, e0, e1);
        *ms = f;
        return true;
    };
    if (cudaMalloc(&sink, blocks * sizeof(float)) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = DWG_ERR_CUDA;
    } else {
        const int it_f = 1 << 16, it_r = 1 << 13;
        double ms_f = 0.0, ms_r = 0.0, ms_e = 0.0, w = 0.0;
        // a short warm-up launch each, then two timed launches each; the
        // shorter time is taken
        bool ok = timed(0, it_f / 8, &w) && timed(1, it_r / 8, &w) && timed(2, it_r / 8, &w);
        double best_f = 1e30, best_r = 1e30, best_e = 1e30;
        for (int r = 0; ok && r < 2; ++r) {
            ok = timed(0, it_f, &ms_f) && timed(1, it_r, &ms_r) && timed(2, it_r, &ms_e);
            best_f = std::min(best_f, ms_f);
            best_r = std::min(best_r, ms_r);
            best_e = std::min(best_e, ms_e);
        }
        if (!ok || cudaGetLastError() != cudaSuccess) {
            rc = DWG_ERR_CUDA;
        } else {
            const double thr = (double)blocks * threads;
            *ffma_lane_ops = thr * it_f * 8.0 * 2.0 / (best_f * 1e-3);
            *rsqrt_ops = thr * it_r * 8.0 / (best_r * 1e-3);
            *ex2_ops = thr * it_r * 8.0 / (best_e * 1e-3);
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    return rc;
}

// ---------------------------------------------------------------------------
// the evaluation kernel
// ---------------------------------------------------------------------------
constexpr int kEvalThreads = 128;  // CTA size of the default shapes
constexpr int kStages = 4;

// One CTA's work: query tile `qtile` against source chunk `chunk`.  With
// CLAMP the records carry delta_j^2 and the kernel is the modified one of
// Sec. 5.2: rho^2 = max(|p_j - q|^2, delta_j^2) (no softening), and inside the
// radius the term's gradient keeps only its -F m / rho^3 part.
template <int P, int NT, bool GRAD, bool SCREENED, bool CLAMP = false, bool COMP = true>
__device__ __forceinline__ void gwn_block(const float *__restrict__ src, int64_t ntiles_total,
                                          const float4 *__restrict__ q, int64_t m,
                                          int tiles_per_chunk, float *__restrict__ part,
                                          int64_t stride, const EvalParams &ep,
                                          int *__restrict__ err, int64_t qtile, int chunk)
{
    constexpr int T = kSrcTile;
    constexpr int RECF = CLAMP ? kSrcFloatsClamp : kSrcFloats;
    constexpr int RQ = RECF / 4;  // 16-byte words per record
    constexpr int TILE_FLOATS = T * RECF;
    constexpr uint32_t TILE_BYTES = TILE_FLOATS * 4;
    constexpr int QB = NT * 2 * P;
    constexpr int NA = GRAD ? 4 : 1;

    __shared__ __align__(128) float sbuf[kStages][TILE_FLOATS];
    __shared__ __align__(8) uint64_t bar[kStages];
    __shared__ int s_abort;

    const int tid = threadIdx.x;
    const int64_t qbase = qtile * QB + tid;
    const int64_t tile0 = (int64_t)chunk * tiles_per_chunk;
    int ntiles = (int)min((int64_t)tiles_per_chunk, ntiles_total - tile0);
    if (ntiles < 0) ntiles = 0;

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&bar[s], 1);
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();
    if (tid == 0) {
        for (int s = 0; s < kStages && s < ntiles; ++s) {
            mbar_expect_tx(&bar[s], TILE_BYTES);
            bulk_g2s(sbuf[s], src + (tile0 + s) * TILE_FLOATS, TILE_BYTES, &bar[s]);
        }
    }

    // query pairs in registers (tail queries repeat the last valid query)
    f2 qx[P], qy[P], qz[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        int64_t i0 = min(qbase + (int64_t)(2 * p) * NT, m - 1);
        int64_t i1 = min(qbase + (int64_t)(2 * p + 1) * NT, m - 1);
        float4 a = q[i0], b = q[i1];
        qx[p] = pk(a.x, b.x);
        qy[p] = pk(a.y, b.y);
        qz[p] = pk(a.z, b.z);
    }
    const f2 eps2 = pk(ep.eps2, ep.eps2);
    const f2 three = pk(3.f, 3.f);
    const f2 zero = pk(0.f, 0.f);
    const f2 sv = pk(ep.s, ep.s);
    const f2 s2v = pk(ep.s2, ep.s2);
    const f2 nl2e = pk(ep.nl2e_s, ep.nl2e_s);

    f2 hw[P], lw[P];
    f2 hgx[P], lgx[P], hgy[P], lgy[P], hgz[P], lgz[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        hw[p] = lw[p] = zero;
        hgx[p] = lgx[p] = hgy[p] = lgy[p] = hgz[p] = lgz[p] = zero;
    }

    int t = 0;
    for (; t < ntiles; ++t) {
        const int s = t % kStages;
        const uint32_t parity = (uint32_t)((t / kStages) & 1);
        if (!mbar_wait_bounded(&bar[s], parity)) {
            atomicOr(err, kErrTimeout);
            s_abort = 1;
        }
        f2 tw[P], t1x[P], t1y[P], t1z[P], t2x[P], t2y[P], t2z[P];
#pragma unroll
        for (int p = 0; p < P; ++p) {
            tw[p] = zero;
            t1x[p] = t1y[p] = t1z[p] = t2x[p] = t2y[p] = t2z[p] = zero;
        }
        if (!s_abort) {
            const ulonglong2 *rec = reinterpret_cast<const ulonglong2 *>(sbuf[s]);
#pragma unroll 2
            for (int j = 0; j < T; ++j) {
                const ulonglong2 r0 = rec[RQ * j + 0];  // (x,x) (y,y)
                const ulonglong2 r1 = rec[RQ * j + 1];  // (z,z) (mx,mx)
                const ulonglong2 r2v = rec[RQ * j + 2]; // (my,my) (mz,mz)
                f2 d2c = zero;
                if (CLAMP) d2c = rec[RQ * j + 3].x;     // (d2,d2)
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    f2 dx = sub2(r0.x, qx[p]);
                    f2 dy = sub2(r0.y, qy[p]);
                    f2 dz = sub2(r1.x, qz[p]);
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
                            tw[p] = add2(tw[p], phi);
                            f2 c = mul2(phi, i2);
                            if (CLAMP) c = keep_ge(c, r2raw, d2c);
                            t1x[p] = fma2(c, dx, t1x[p]);
                            t1y[p] = fma2(c, dy, t1y[p]);
                            t1z[p] = fma2(c, dz, t1z[p]);
                            t2x[p] = fma2(r1.y, i3, t2x[p]);
                            t2y[p] = fma2(r2v.x, i3, t2y[p]);
                            t2z[p] = fma2(r2v.y, i3, t2z[p]);
                        } else {
                            tw[p] = fma2(md, i3, tw[p]);
                        }
                    } else {
                        // g = F / rho^3 = e^(-s rho) (1 + s rho) / rho^3
                        //   = e inv^2 (inv + s)
                        f2 rho = mul2(rr, inv);
                        f2 e = ex22(mul2(rho, nl2e));
                        f2 g = mul2(mul2(i2, add2(inv, sv)), e);
                        tw[p] = fma2(g, md, tw[p]);
                        if (GRAD) {
                            // md (3 F / rho^5 + s^2 e / rho^3)
                            //   = md inv^2 (3 g + s^2 e inv)
                            f2 cc = fma2(three, g, mul2(e, mul2(s2v, inv)));
                            f2 c = mul2(md, mul2(i2, cc));
                            if (CLAMP) c = keep_ge(c, r2raw, d2c);
                            t1x[p] = fma2(c, dx, t1x[p]);
                            t1y[p] = fma2(c, dy, t1y[p]);
                            t1z[p] = fma2(c, dz, t1z[p]);
                            t2x[p] = fma2(r1.y, g, t2x[p]);
                            t2y[p] = fma2(r2v.x, g, t2y[p]);
                            t2z[p] = fma2(r2v.y, g, t2z[p]);
                        }
                    }
                }
            }
        }
        // fold the tile sums into the compensated totals (COMP false: plain
        // FP32 addition, the uncompensated form kept for precision studies)
#pragma unroll
        for (int p = 0; p < P; ++p) {
            if (COMP) two_sum_acc(hw[p], lw[p], tw[p]);
            else hw[p] = add2(hw[p], tw[p]);
            if (GRAD) {
                f2 gx, gy, gz;
                if (!SCREENED) {
                    gx = sub2(mul2(three, t1x[p]), t2x[p]);
                    gy = sub2(mul2(three, t1y[p]), t2y[p]);
                    gz = sub2(mul2(three, t1z[p]), t2z[p]);
                } else {
                    gx = sub2(t1x[p], t2x[p]);
                    gy = sub2(t1y[p], t2y[p]);
                    gz = sub2(t1z[p], t2z[p]);
                }
                if (COMP) {
                    two_sum_acc(hgx[p], lgx[p], gx);
                    two_sum_acc(hgy[p], lgy[p], gy);
                    two_sum_acc(hgz[p], lgz[p], gz);
                } else {
                    hgx[p] = add2(hgx[p], gx);
                    hgy[p] = add2(hgy[p], gy);
                    hgz[p] = add2(hgz[p], gz);
                }
            }
        }
        __syncthreads();  // every thread is done with buffer s
        if (s_abort) break;
        if (tid == 0 && t + kStages < ntiles) {
            mbar_expect_tx(&bar[s], TILE_BYTES);
            bulk_g2s(sbuf[s], src + (tile0 + t + kStages) * TILE_FLOATS, TILE_BYTES, &bar[s]);
        }
    }
    if (s_abort) {
        // drain the copies still in flight before the CTA's shared memory goes
        // away, the one whose wait gave up (tile t) included
        if (tid == 0)
            for (int u = t; u < ntiles && u < t + kStages; ++u)
                mbar_wait_bounded(&bar[u % kStages], (uint32_t)((u / kStages) & 1));
        __syncthreads();
    }

    // write the (hi, lo) partials: part[((chunk * NA + a) * 2 + h) * stride + i]
#pragma unroll
    for (int p = 0; p < P; ++p) {
#pragma unroll
        for (int lane = 0; lane < 2; ++lane) {
            int64_t i = qbase + (int64_t)(2 * p + lane) * NT;
            if (i >= m) continue;
            float vals[NA][2];
            float a, b;
            upk(hw[p], a, b);
            vals[0][0] = lane ? b : a;
            upk(lw[p], a, b);
            vals[0][1] = lane ? b : a;
            if (GRAD) {
                upk(hgx[p], a, b); vals[1 % NA][0] = lane ? b : a;
                upk(lgx[p], a, b); vals[1 % NA][1] = lane ? b : a;
                upk(hgy[p], a, b); vals[2 % NA][0] = lane ? b : a;
                upk(lgy[p], a, b); vals[2 % NA][1] = lane ? b : a;
                upk(hgz[p], a, b); vals[3 % NA][0] = lane ? b : a;
                upk(lgz[p], a, b); vals[3 % NA][1] = lane ? b : a;
            }
#pragma unroll
            for (int aa = 0; aa < NA; ++aa)
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    part[((int64_t)(chunk * NA + aa) * 2 + h) * stride + i] = vals[aa][h];
        }
    }
}

template <int P, int NT, bool GRAD, bool SCREENED, bool CLAMP = false, bool COMP = true>
__global__ void __launch_bounds__(NT)
    k_gwn(const float *__restrict__ src, int64_t ntiles_total, const float4 *__restrict__ q,
          int64_t m, int tiles_per_chunk, float *__restrict__ part, int64_t stride,
          EvalParams ep, int *__restrict__ err)
{
    gwn_block<P, NT, GRAD, SCREENED, CLAMP, COMP>(src, ntiles_total, q, m, tiles_per_chunk,
                                                  part, stride, ep, err, (int64_t)blockIdx.x,
                                                  (int)blockIdx.y);
}

// Many clouds in one launch: CTA b runs work item items[b] of its cloud;
// clouds that have converged are skipped.
template <int P, bool GRAD, bool SCREENED>
__global__ void __launch_bounds__(kEvalThreads)
    k_gwn_batch(const GwnCloud *__restrict__ clouds, const GwnItem *__restrict__ items,
                int *__restrict__ err)
{
    const GwnItem it = items[blockIdx.x];
    const GwnCloud &C = clouds[it.cloud];
    if (C.st && cloud_idle(C.st)) return;
    gwn_block<P, kEvalThreads, GRAD, SCREENED>(C.src, C.ntiles, C.q, C.m, C.tpc, C.part, C.stride,
                                               C.ep, err, (int64_t)it.qtile, it.chunk);
}

// ---------------------------------------------------------------------------
// source records: (x,x,y,y,z,z,mx,mx,my,my,mz,mz), m = a n / (4 pi);
// padding records are at the origin with m = 0 and contribute exactly 0.
// ---------------------------------------------------------------------------
__global__ void k_pack_sources(const float4 *__restrict__ p4, const float4 *__restrict__ nrm,
                               int64_t n, int64_t npad, float *__restrict__ src)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npad) return;
    float x = 0.f, y = 0.f, z = 0.f, mx = 0.f, my = 0.f, mz = 0.f;
    if (i < n) {
        float4 p = p4[i];
        float4 v = nrm[i];
        float c = p.w * (float)(1.0 / (4.0 * kPi));
        x = p.x; y = p.y; z = p.z;
        mx = c * v.x; my = c * v.y; mz = c * v.z;
    }
    float4 *r = reinterpret_cast<float4 *>(src + i * kSrcFloats);
    r[0] = make_float4(x, x, y, y);
    r[1] = make_float4(z, z, mx, mx);
    r[2] = make_float4(my, my, mz, mz);
}

// records of the modified kernel: the 12 floats above and (d2,d2,0,0);
// padding records get d2 = 1 (with m = 0 they still contribute exactly 0)
__global__ void k_pack_sources16(const float4 *__restrict__ p4, const float4 *__restrict__ nrm,
                                 const float *__restrict__ delta2, int64_t n, int64_t npad,
                                 float *__restrict__ src)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npad) return;
    float x = 0.f, y = 0.f, z = 0.f, mx = 0.f, my = 0.f, mz = 0.f, d2 = 1.f;
    if (i < n) {
        float4 p = p4[i];
        float4 v = nrm[i];
        float c = p.w * (float)(1.0 / (4.0 * kPi));
        x = p.x; y = p.y; z = p.z;
        mx = c * v.x; my = c * v.y; mz = c * v.z;
        d2 = delta2[i];
    }
    float4 *r = reinterpret_cast<float4 *>(src + i * kSrcFloatsClamp);
    r[0] = make_float4(x, x, y, y);
    r[1] = make_float4(z, z, mx, mx);
    r[2] = make_float4(my, my, mz, mz);
    r[3] = make_float4(d2, d2, 0.f, 0.f);
}

cudaError_t launch_pack_sources16(const Ctx *c)
{
    k_pack_sources16<<<(unsigned)ceil_div(c->npad, 256), 256, 0, c->stream>>>(
        c->d_p4, c->d_nrm, c->d_delta2, c->n, c->npad, c->d_src16);
    return cudaGetLastError();
}

cudaError_t launch_pack_sources(const float4 *p4, const float4 *nrm, int64_t n, int64_t npad,
                                float *src, cudaStream_t s)
{
    int blk = 256;
    k_pack_sources<<<(unsigned)ceil_div(npad, blk), blk, 0, s>>>(p4, nrm, n, npad, src);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
EvalParams make_eval_params(const Ctx *c)
{
    EvalParams ep;
    ep.eps2 = c->reg_mode == DWG_REG_CLAMP ? 0.f : c->eps * c->eps;
    bool scr = c->kernel == DWG_KERNEL_SCREENED && c->lambda > 0.f;
    ep.screened = scr ? 1 : 0;
    double s = scr ? sqrt((double)c->lambda) : 0.0;
    ep.s = (float)s;
    ep.s2 = (float)(s * s);
    ep.nl2e_s = (float)(-s * 1.4426950408889634);
    return ep;
}

static int num_sms(int dev)
{
    static int cached[64] = {0};
    if (dev < 0 || dev >= 64) return 148;
    if (!cached[dev]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = v > 0 ? v : 148;
    }
    return cached[dev];
}

// Split the sources into chunks so that the grid fills the GPU in whole
// waves: with `slots` resident CTAs, a grid of qtiles * ch CTAs of
// ceil(ntiles / ch) tiles each takes ceil(qtiles * ch / slots) waves; pick
// the chunk count with the smallest waves * tiles-per-chunk (fewest chunks
// on ties), each chunk keeping at least 8 tiles.
static int pick_chunks(int64_t qtiles, int64_t ntiles_src, int slots)
{
    if (qtiles < 1) qtiles = 1;
    if (slots < 1) slots = 1;
    int64_t maxch = ntiles_src / 8;
    if (maxch < 1) maxch = 1;
    if (maxch > 64) maxch = 64;
    int best = 1;
    int64_t best_cost = INT64_MAX;
    for (int64_t ch = 1; ch <= maxch; ++ch) {
        int64_t tpc = ceil_div(ntiles_src, ch);
        int64_t waves = ceil_div(qtiles * ch, slots);
        int64_t cost = waves * tpc;
        if (cost < best_cost) {
            best_cost = cost;
            best = (int)ch;
        }
    }
    return best;
}

// ---------------------------------------------------------------------------
// evaluator shapes: (query pairs per thread P, CTA size NT); the tuner picks
// one per kind (w and gradient at the points, w only at the corners)
// ---------------------------------------------------------------------------
typedef void (*GwnKernel)(const float *, int64_t, const float4 *, int64_t, int, float *, int64_t,
                          EvalParams, int *);
struct GwnVariant {
    int p, nt;
    GwnKernel k[2];  // plain, screened
};
#define DWG_GWN_VARIANT(P, NT, G) \
    {P, NT, {k_gwn<P, NT, G, false>, k_gwn<P, NT, G, true>}}
static const GwnVariant kVarGrad[] = {
    DWG_GWN_VARIANT(2, 128, true), DWG_GWN_VARIANT(1, 128, true), DWG_GWN_VARIANT(3, 128, true),
    DWG_GWN_VARIANT(1, 256, true), DWG_GWN_VARIANT(2, 256, true)};
static const GwnVariant kVarW[] = {
    DWG_GWN_VARIANT(4, 128, false), DWG_GWN_VARIANT(2, 128, false), DWG_GWN_VARIANT(3, 128, false),
    DWG_GWN_VARIANT(6, 128, false), DWG_GWN_VARIANT(2, 256, false), DWG_GWN_VARIANT(3, 256, false),
    DWG_GWN_VARIANT(4, 256, false), DWG_GWN_VARIANT(1, 128, false), DWG_GWN_VARIANT(1, 256, false),
    DWG_GWN_VARIANT(2, 64, false)};
#undef DWG_GWN_VARIANT
// the modified kernel runs in the default shapes only
static const GwnVariant kVarClampGrad = {2, 128, {k_gwn<2, 128, true, false, true>,
                                                  k_gwn<2, 128, true, true, true>}};
static const GwnVariant kVarClampW = {4, 128, {k_gwn<4, 128, false, false, true>,
                                               k_gwn<4, 128, false, true, true>}};
// the uncompensated fold (precision studies), default shapes only
static const GwnVariant kVarPlainFoldGrad = {2, 128, {k_gwn<2, 128, true, false, false, false>,
                                                      k_gwn<2, 128, true, true, false, false>}};
static const GwnVariant kVarPlainFoldW = {4, 128, {k_gwn<4, 128, false, false, false, false>,
                                                   k_gwn<4, 128, false, true, false, false>}};
constexpr int kNumVarGrad = (int)(sizeof(kVarGrad) / sizeof(kVarGrad[0]));
constexpr int kNumVarW = (int)(sizeof(kVarW) / sizeof(kVarW[0]));

int eval_variant_count(bool grad) { return grad ? kNumVarGrad : kNumVarW; }

void eval_variant_shape(bool grad, int v, int *p, int *nt)
{
    const GwnVariant &V = grad ? kVarGrad[v] : kVarW[v];
    *p = V.p;
    *nt = V.nt;
}

static const GwnVariant &variant(bool grad, int v)
{
    if (grad) return kVarGrad[(v >= 0 && v < kNumVarGrad) ? v : 0];
    return kVarW[(v >= 0 && v < kNumVarW) ? v : 0];
}

// variant v of the context's kernel (the modified kernel and the
// uncompensated fold have one shape each)
static const GwnVariant &variant_of(const Ctx *c, bool grad, int v)
{
    if (c->reg_mode == DWG_REG_CLAMP) return grad ? kVarClampGrad : kVarClampW;
    if (!c->compensated) return grad ? kVarPlainFoldGrad : kVarPlainFoldW;
    return variant(grad, v);
}

// occupancy-cache slot of a context's variant
static int slot_of(const Ctx *c, int v)
{
    if (c->reg_mode == DWG_REG_CLAMP) return 15;
    if (!c->compensated) return 14;
    return v;
}

// resident CTAs of a variant on the whole device (cached per device; the
// modified kernel's shape in slot 15)
static int variant_slots(const GwnVariant &V, bool grad, int v, bool scr, int dev)
{
    static int cached[2][2][16][64] = {};
    if (dev < 0 || dev >= 64) dev = 0;
    if (v < 0 || v >= 16) v = 0;
    int &slot = cached[grad][scr][v][dev];
    if (!slot) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, V.k[scr ? 1 : 0], V.nt, 0) !=
                cudaSuccess ||
            nb < 1) {
            cudaGetLastError();
            nb = 1;
        }
        slot = nb * num_sms(dev);
    }
    return slot;
}

static bool screened_of(const Ctx *c) { return c->kernel == DWG_KERNEL_SCREENED && c->lambda > 0.f; }

int eval_chunks_variant(const Ctx *c, int64_t m, bool grad, int v)
{
    const GwnVariant &V = variant_of(c, grad, v);
    const int slot_id = slot_of(c, v);
    int64_t QB = (int64_t)V.nt * 2 * V.p;
    return pick_chunks(ceil_div(m, QB), c->npad / kSrcTile,
                       variant_slots(V, grad, slot_id, screened_of(c), c->device));
}

int eval_chunks(const Ctx *c, int64_t m, bool grad)
{
    return eval_chunks_variant(c, m, grad, grad ? c->var_grad : c->var_w);
}

int eval_launch_variant(Ctx *c, const float4 *q, int64_t m, bool grad, int v, int nchunks,
                        float *part, int64_t stride)
{
    const GwnVariant &V = variant_of(c, grad, v);
    EvalParams ep = make_eval_params(c);
    int64_t QB = (int64_t)V.nt * 2 * V.p;
    int64_t qtiles = ceil_div(m, QB);
    int64_t ntiles = c->npad / kSrcTile;
    int tpc = (int)ceil_div(ntiles, nchunks);
    dim3 grid((unsigned)qtiles, (unsigned)nchunks);
    const float *src = c->reg_mode == DWG_REG_CLAMP ? c->d_src16 : c->d_src;
    V.k[ep.screened ? 1 : 0]<<<grid, V.nt, 0, c->stream>>>(src, ntiles, q, m, tpc, part, stride,
                                                             ep, c->d_err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        c->err = std::string("gwn kernel launch: ") + cudaGetErrorString(e);
        return DWG_ERR_CUDA;
    }
    return DWG_OK;
}

int eval_launch(Ctx *c, const float4 *q, int64_t m, bool grad, int nchunks, float *part,
                int64_t stride)
{
    return eval_launch_variant(c, q, m, grad, grad ? c->var_grad : c->var_w, nchunks, part,
                               stride);
}

constexpr int kPGrad = 2;   // query pairs per thread, gradient kernel (batched launches)
constexpr int kPW = 4;      // query pairs per thread, w-only kernel (batched and raw launches)

// ---------------------------------------------------------------------------
// reduce: combine chunk partials in chunk order; for gradients add back the
// coincident-source terms; optionally per-block FP64 sums of w.
// ---------------------------------------------------------------------------
template <bool GRAD>
__device__ __forceinline__ void reduce_points_body(const float *__restrict__ part, int nchunks,
                                                   int64_t m, int64_t stride,
                                                   const float4 *__restrict__ q,
                                                   const float *__restrict__ src, int rec_floats,
                                                   const uint64_t *__restrict__ codes,
                                                   int64_t nsrc, int self_mode, const CubeQ &cq,
                                                   const EvalParams &ep, float4 *__restrict__ out,
                                                   double *__restrict__ wsum_blocks, int64_t bid)
{
    constexpr int NA = GRAD ? 4 : 1;
    int64_t i = bid * blockDim.x + threadIdx.x;
    double wloc = 0.0;
    if (i < m) {
        float h[NA], l[NA];
        for (int a = 0; a < NA; ++a) { h[a] = 0.f; l[a] = 0.f; }
        for (int ch = 0; ch < nchunks; ++ch)
            for (int a = 0; a < NA; ++a) {
                float ph = part[((int64_t)(ch * NA + a) * 2 + 0) * stride + i];
                float pl = part[((int64_t)(ch * NA + a) * 2 + 1) * stride + i];
                two_sum1(h[a], l[a], ph);
                l[a] = __fadd_rn(l[a], pl);
            }
        if (GRAD && self_mode != 0) {
            // The coincident sources' gradient term is -(F inv^3) m with
            // rho = eps; add it back so that those sources are skipped
            // (the factor rounded as the evaluators round it).
            float4 qi = q[i];
            auto factor = [&](float rr) {
                const float inv = rsqrt_mufu(rr);
                const float i2 = inv * inv;
                if (!ep.screened) return i2 * inv;
                const float e = ex2_mufu((rr * inv) * ep.nl2e_s);
                return (i2 * (inv + ep.s)) * e;
            };
            float fi3 = factor(ep.eps2);
            int64_t lo_j, hi_j;
            if (self_mode == 1) {  // queries are the sources, same order
                lo_j = i;
                hi_j = i + 1;
                uint64_t ci = codes[i];
                while (lo_j > 0 && codes[lo_j - 1] == ci) --lo_j;
                while (hi_j < nsrc && codes[hi_j] == ci) ++hi_j;
            } else {  // arbitrary query: locate its code among the sorted codes
                uint64_t ci = spread3((uint64_t)quant21(qi.x, cq.lo[0], cq.inv_h21)) |
                              (spread3((uint64_t)quant21(qi.y, cq.lo[1], cq.inv_h21)) << 1) |
                              (spread3((uint64_t)quant21(qi.z, cq.lo[2], cq.inv_h21)) << 2);
                int64_t a = 0, b = nsrc;
                while (a < b) {
                    int64_t mid = (a + b) >> 1;
                    if (codes[mid] < ci) a = mid + 1; else b = mid;
                }
                lo_j = a;
                hi_j = a;
                while (hi_j < nsrc && codes[hi_j] == ci) ++hi_j;
            }
            for (int64_t j = lo_j; j < hi_j; ++j) {
                const float *r = src + j * rec_floats;
                if (r[0] == qi.x && r[2] == qi.y && r[4] == qi.z) {
                    if (rec_floats == kSrcFloatsClamp) {
                        // modified kernel: this source's rho is its own delta_j
                        fi3 = factor(r[12]);
                    }
                    two_sum1(h[1], l[1], r[6] * fi3);
                    two_sum1(h[2], l[2], r[8] * fi3);
                    two_sum1(h[3], l[3], r[10] * fi3);
                }
            }
        }
        float w = __fadd_rn(h[0], l[0]);
        float4 o = make_float4(0.f, 0.f, 0.f, w);
        if (GRAD) {
            o.x = __fadd_rn(h[1], l[1]);
            o.y = __fadd_rn(h[2], l[2]);
            o.z = __fadd_rn(h[3], l[3]);
        }
        out[i] = o;
        wloc = (double)h[0] + (double)l[0];
    }
    if (wsum_blocks) {
        // deterministic block sum of w in FP64 (fixed tree)
        __shared__ double sh[256];
        sh[threadIdx.x] = wloc;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) wsum_blocks[bid] = sh[0];
    }
}

template <bool GRAD>
__global__ void k_reduce_points(const float *__restrict__ part, int nchunks, int64_t m,
                                int64_t stride, const float4 *__restrict__ q,
                                const float *__restrict__ src, int rec_floats,
                                const uint64_t *__restrict__ codes, int64_t nsrc, int self_mode,
                                CubeQ cq, EvalParams ep, float4 *__restrict__ out,
                                double *__restrict__ wsum_blocks)
{
    reduce_points_body<GRAD>(part, nchunks, m, stride, q, src, rec_floats, codes, nsrc,
                             self_mode, cq, ep, out, wsum_blocks, blockIdx.x);
}

int wsum_block_count(int64_t n) { return (int)ceil_div(n, 256); }

__device__ __forceinline__ void reduce_w_body(const float *__restrict__ part, int nchunks,
                                              int64_t m, int64_t stride, float *__restrict__ out,
                                              int64_t bid)
{
    int64_t i = bid * blockDim.x + threadIdx.x;
    if (i >= m) return;
    float h = 0.f, l = 0.f;
    for (int ch = 0; ch < nchunks; ++ch) {
        two_sum1(h, l, part[((int64_t)ch * 2 + 0) * stride + i]);
        l = __fadd_rn(l, part[((int64_t)ch * 2 + 1) * stride + i]);
    }
    out[i] = __fadd_rn(h, l);
}

__global__ void k_reduce_w(const float *__restrict__ part, int nchunks, int64_t m, int64_t stride,
                           float *__restrict__ out)
{
    reduce_w_body(part, nchunks, m, stride, out, blockIdx.x);
}

// batched: every cloud of a batch in one launch (the point reduce of a
// batch runs with self_mode 1 and the gradient, as each cloud's own launch)
__global__ void k_reduce_points_b(const CloudIter *__restrict__ cl, const int *__restrict__ off,
                                  int ncl)
{
    const int ci = seg_cloud(off, ncl);
    const CloudIter &c = cl[ci];
    reduce_points_body<true>(c.part_p, c.nchunks_p, c.n, c.n, c.p4, c.src, kSrcFloats, c.codes,
                             c.n, 1, c.cq, c.ep, c.wg, c.wsum_blocks,
                             (int64_t)blockIdx.x - off[ci]);
}

__global__ void k_reduce_w_b(const CloudIter *__restrict__ cl, const int *__restrict__ off, int ncl)
{
    const int ci = seg_cloud(off, ncl);
    const CloudIter &c = cl[ci];
    reduce_w_body(c.part_c, c.nchunks_c, c.ncorners, c.ncorners, c.wc,
                  (int64_t)blockIdx.x - off[ci]);
}

cudaError_t launch_eval_batch(int phase, const CloudIter *cl, const int *off, int ncl,
                              int blocks, cudaStream_t s)
{
    if (blocks <= 0) return cudaSuccess;
    if (phase == kPhReducePoints)
        k_reduce_points_b<<<(unsigned)blocks, 256, 0, s>>>(cl, off, ncl);
    else if (phase == kPhReduceW)
        k_reduce_w_b<<<(unsigned)blocks, 256, 0, s>>>(cl, off, ncl);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_reduce_w(Ctx *c, const float *part, int nchunks, int64_t m, float *out)
{
    k_reduce_w<<<(unsigned)ceil_div(m, 256), 256, 0, c->stream>>>(part, nchunks, m, m, out);
    return cudaGetLastError();
}

cudaError_t launch_reduce_points(Ctx *c, const float *part, int nchunks, int64_t m,
                                 const float4 *queries, int self_mode, bool grad,
                                 float4 *out, double *wsum_blocks)
{
    CubeQ cq;
    for (int k = 0; k < 3; ++k) cq.lo[k] = c->cube_lo[k];
    cq.inv_h21 = (double)(1 << kMortonBits) / c->cube_L;
    EvalParams ep = make_eval_params(c);
    unsigned blocks = (unsigned)ceil_div(m, 256);
    const bool clamp = c->reg_mode == DWG_REG_CLAMP;
    const float *src = clamp ? c->d_src16 : c->d_src;
    const int recf = clamp ? kSrcFloatsClamp : kSrcFloats;
    if (grad)
        k_reduce_points<true><<<blocks, 256, 0, c->stream>>>(part, nchunks, m, m, queries, src,
                                                             recf, c->d_codes, c->n, self_mode,
                                                             cq, ep, out, wsum_blocks);
    else
        k_reduce_points<false><<<blocks, 256, 0, c->stream>>>(part, nchunks, m, m, queries, src,
                                                              recf, c->d_codes, c->n, 0, cq, ep,
                                                              out, wsum_blocks);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// launchers without an engine context (caller-provided buffers)
// ---------------------------------------------------------------------------
int gwn_w_chunks_raw(int64_t m, int64_t npad, int device)
{
    return pick_chunks(ceil_div(m, kEvalThreads * 2 * kPW), npad / kSrcTile,
                       variant_slots(kVarW[0], false, 0, false, device));
}

cudaError_t launch_gwn_w_raw(const float *src, int64_t npad, const float4 *q, int64_t m,
                             int nchunks, float *part, const EvalParams &ep, int *err,
                             cudaStream_t s)
{
    constexpr int QB = kEvalThreads * 2 * kPW;
    int64_t ntiles = npad / kSrcTile;
    int tpc = (int)ceil_div(ntiles, nchunks);
    dim3 grid((unsigned)ceil_div(m, QB), (unsigned)nchunks);
    if (ep.screened)
        k_gwn<kPW, kEvalThreads, false, true>
            <<<grid, kEvalThreads, 0, s>>>(src, ntiles, q, m, tpc, part, m, ep, err);
    else
        k_gwn<kPW, kEvalThreads, false, false>
            <<<grid, kEvalThreads, 0, s>>>(src, ntiles, q, m, tpc, part, m, ep, err);
    return cudaGetLastError();
}

cudaError_t launch_reduce_w_raw(const float *part, int nchunks, int64_t m, float *out,
                                cudaStream_t s)
{
    k_reduce_w<<<(unsigned)ceil_div(m, 256), 256, 0, s>>>(part, nchunks, m, m, out);
    return cudaGetLastError();
}

int batch_query_tile(bool grad) { return kEvalThreads * 2 * (grad ? kPGrad : kPW); }

cudaError_t launch_gwn_batch(const GwnCloud *clouds, const GwnItem *items, int64_t nitems,
                             bool grad, bool screened, int *err, cudaStream_t s)
{
    if (nitems <= 0) return cudaSuccess;
    unsigned g = (unsigned)nitems;
    if (grad) {
        if (screened) k_gwn_batch<kPGrad, true, true><<<g, kEvalThreads, 0, s>>>(clouds, items, err);
        else k_gwn_batch<kPGrad, true, false><<<g, kEvalThreads, 0, s>>>(clouds, items, err);
    } else {
        if (screened) k_gwn_batch<kPW, false, true><<<g, kEvalThreads, 0, s>>>(clouds, items, err);
        else k_gwn_batch<kPW, false, false><<<g, kEvalThreads, 0, s>>>(clouds, items, err);
    }
    return cudaGetLastError();
}

}  // namespace dwg
