// dwg_noalloc.cu -- w evaluation for callers that cannot allocate device
// memory.
//
// Some callers own every byte of device memory through their own pool and a
// fixed budget (a serving process that reserves HBM up front, an embedding
// framework with its own allocator), and some cannot afford cudaMalloc or
// cudaFree in the middle of their work: cudaFree synchronises the whole
// device, and an allocation can fail at an arbitrary point of a run.  The
// handle-based entry points allocate their work buffers; this entry point
// does not.  Its scratch -- the packed source records, the query records, the
// per-chunk partial sums and an error word -- lives in one file-scope
// __device__ array of fixed size, which every GPU that loads the library
// keeps until the process exits.
#include <mutex>
#include <string>

#include "dwg_internal.cuh"

namespace dwg {

constexpr int64_t kNoAllocMaxPoints = 65536;    // sources
constexpr int64_t kNoAllocMaxQueries = 262144;  // query points
constexpr size_t kNoAllocErrBytes = 256;
constexpr size_t kNoAllocSrcBytes = (size_t)kNoAllocMaxPoints * kSrcFloats * sizeof(float);
constexpr size_t kNoAllocQryBytes = (size_t)kNoAllocMaxQueries * sizeof(float4);
constexpr size_t kNoAllocPartBytes = (size_t)8 << 20;
constexpr size_t kNoAllocBytes =
    kNoAllocErrBytes + kNoAllocSrcBytes + kNoAllocQryBytes + kNoAllocPartBytes;  // 15 MiB + 256 B

// The scratch.  Host code must not use this name as an address: it is a
// host-side stand-in.  The device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

static std::mutex g_noalloc_mu;
static void *g_noalloc_ptr[64];

// failures are reported through dwg_last_error(NULL)
static int noalloc_fail(int code, const std::string &msg)
{
    set_global_error(msg);
    return code;
}

// Device address of the scratch on the current device, looked up once per
// device (with that device current) and cached.
static int noalloc_scratch(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= 64) return noalloc_fail(DWG_ERR_INVALID, "device index out of range");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_global_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return DWG_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_noalloc_ptr[dev]);
    return DWG_OK;
}

// source records (x,x,y,y,z,z,mx,mx,my,my,mz,mz), m = a n / (4 pi), normals
// normalised; padding records at the origin with m = 0
__global__ void k_noalloc_pack(const float *__restrict__ xyz, const float *__restrict__ nrm,
                               const float *__restrict__ a, int64_t n, int64_t npad,
                               float *__restrict__ src, int *err)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npad) return;
    float x = 0.f, y = 0.f, z = 0.f, mx = 0.f, my = 0.f, mz = 0.f;
    if (i < n) {
        x = xyz[3 * i]; y = xyz[3 * i + 1]; z = xyz[3 * i + 2];
        float vx = nrm[3 * i], vy = nrm[3 * i + 1], vz = nrm[3 * i + 2];
        float l = sqrtf(vx * vx + vy * vy + vz * vz);
        float w = a ? a[i] : 1.f;
        if (!(l > 0.f) || !isfinite(l) || !isfinite(x) || !isfinite(y) || !isfinite(z) ||
            !(w > 0.f) || !isfinite(w)) {
            atomicOr(err, kErrNonfinite);
            l = 1.f;
        }
        float c = w * (float)(1.0 / (4.0 * kPi));
        mx = c * (vx / l); my = c * (vy / l); mz = c * (vz / l);
    }
    float4 *r = reinterpret_cast<float4 *>(src + i * kSrcFloats);
    r[0] = make_float4(x, x, y, y);
    r[1] = make_float4(z, z, mx, mx);
    r[2] = make_float4(my, my, mz, mz);
}

__global__ void k_noalloc_queries(const float *__restrict__ v, int64_t m, float4 *out, int *err)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    float x = v[3 * i], y = v[3 * i + 1], z = v[3 * i + 2];
    if (!isfinite(x) || !isfinite(y) || !isfinite(z)) atomicOr(err, kErrNonfinite);
    out[i] = make_float4(x, y, z, 0.f);
}

// true for managed memory and for device memory of device `dev`; a pointer
// into another GPU's memory is refused (without peer access the kernels below
// could not read it)
static bool on_device(const void *p, int dev)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace dwg

using namespace dwg;

extern "C" int dwg_eval_w_noalloc(const float *points, const float *normals, const float *weights,
                                  int64_t n, const float *queries, int64_t m, int kernel,
                                  float eps, float screening, float *w_out, void *stream)
{
    if (!points || !normals || !queries || !w_out)
        return noalloc_fail(DWG_ERR_INVALID, "dwg_eval_w_noalloc: null pointer");
    if (n < 1 || n > kNoAllocMaxPoints)
        return noalloc_fail(DWG_ERR_INVALID,
                            "dwg_eval_w_noalloc: n must be in [1, 65536] (fixed scratch size)");
    if (m < 1 || m > kNoAllocMaxQueries)
        return noalloc_fail(DWG_ERR_INVALID,
                            "dwg_eval_w_noalloc: m must be in [1, 262144] (fixed scratch size)");
    if (kernel != DWG_KERNEL_PLAIN && kernel != DWG_KERNEL_SCREENED)
        return noalloc_fail(DWG_ERR_INVALID, "dwg_eval_w_noalloc: unknown kernel");
    if (!(eps > 0.f) || !isfinite(eps) || !(screening >= 0.f) || !isfinite(screening))
        return noalloc_fail(DWG_ERR_INVALID, "dwg_eval_w_noalloc: need eps > 0, screening >= 0");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(DWG_ERR_CUDA, cudaGetErrorString(e));
    if (!on_device(points, dev) || !on_device(normals, dev) || !on_device(queries, dev) ||
        !on_device(w_out, dev) || (weights && !on_device(weights, dev)))
        return noalloc_fail(DWG_ERR_INVALID,
                            "dwg_eval_w_noalloc: every array must be device memory of the "
                            "current device");
    unsigned char *base = nullptr;
    int rc = noalloc_scratch(dev, &base);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    int *err = reinterpret_cast<int *>(base);
    float *src = reinterpret_cast<float *>(base + kNoAllocErrBytes);
    float4 *q4 = reinterpret_cast<float4 *>(base + kNoAllocErrBytes + kNoAllocSrcBytes);
    float *part =
        reinterpret_cast<float *>(base + kNoAllocErrBytes + kNoAllocSrcBytes + kNoAllocQryBytes);

    const int64_t npad = ceil_div(n, kSrcTile) * kSrcTile;
    int nchunks = gwn_w_chunks_raw(m, npad, dev);
    int64_t cap = (int64_t)(kNoAllocPartBytes / (2 * sizeof(float) * (size_t)m));
    if (nchunks > cap) nchunks = (int)cap;
    if (nchunks < 1) nchunks = 1;

    EvalParams ep;
    ep.eps2 = eps * eps;
    bool scr = kernel == DWG_KERNEL_SCREENED && screening > 0.f;
    ep.screened = scr ? 1 : 0;
    double sq = scr ? sqrt((double)screening) : 0.0;
    ep.s = (float)sq;
    ep.s2 = (float)(sq * sq);
    ep.nl2e_s = (float)(-sq * 1.4426950408889634);

    // the error word starts at zero on every call; every other scratch byte
    // that is read is written first by this call
    if ((e = cudaMemsetAsync(err, 0, sizeof(int), s)) != cudaSuccess)
        return noalloc_fail(DWG_ERR_CUDA, cudaGetErrorString(e));
    k_noalloc_pack<<<(unsigned)ceil_div(npad, 256), 256, 0, s>>>(points, normals, weights, n, npad,
                                                                  src, err);
    k_noalloc_queries<<<(unsigned)ceil_div(m, 256), 256, 0, s>>>(queries, m, q4, err);
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = launch_gwn_w_raw(src, npad, q4, m, nchunks, part, ep, err, s)) != cudaSuccess ||
        (e = launch_reduce_w_raw(part, nchunks, m, w_out, s)) != cudaSuccess)
        return noalloc_fail(DWG_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    int herr = 0;
    if ((e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return noalloc_fail(DWG_ERR_CUDA, cudaGetErrorString(e));
    if (herr & kErrTimeout) return noalloc_fail(DWG_ERR_TIMEOUT, "a device-side wait gave up");
    if (herr & kErrNonfinite)
        return noalloc_fail(DWG_ERR_NONFINITE,
                            "non-finite input, zero normal or non-positive weight");
    if (herr) return noalloc_fail(DWG_ERR_CUDA, "device error flag set");
    return DWG_OK;
}
