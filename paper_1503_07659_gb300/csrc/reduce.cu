// FP64 reductions on the GPU for residual and energy checks of the mixed
// precision forms: max|a-b|, max|b| and the dot product a.b, every operand
// widened to double first.  Two passes with a fixed partition (per-block
// partials in caller workspace, then one block), so the result is the same on
// every call with the same count.
#include <cuda.h>

#include <mutex>

#include "common.cuh"

namespace semax {

constexpr int kRedThreads = 256;
constexpr int kRedMaxBlocks = 1024;

static int reduce_blocks(int64_t count) {
    int64_t b = (count + kRedThreads * 8 - 1) / (kRedThreads * 8);
    if (b < 1) b = 1;
    if (b > kRedMaxBlocks) b = kRedMaxBlocks;
    return (int)b;
}

// max that keeps a NaN once one is seen
__device__ __forceinline__ double nan_max(double a, double b) {
    return (a != a) ? a : ((b != b || b > a) ? b : a);
}

// Block-wide reduction of (m0, m1, s) in a fixed order; result in thread 0.
__device__ __forceinline__ void block_reduce3(double &m0, double &m1, double &s) {
    __shared__ double sh[3][kRedThreads / 32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        m0 = nan_max(m0, __shfl_down_sync(0xffffffffu, m0, off));
        m1 = nan_max(m1, __shfl_down_sync(0xffffffffu, m1, off));
        s += __shfl_down_sync(0xffffffffu, s, off);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sh[0][warp] = m0; sh[1][warp] = m1; sh[2][warp] = s; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < kRedThreads / 32; ++q) {
            m0 = nan_max(m0, sh[0][q]);
            m1 = nan_max(m1, sh[1][q]);
            s += sh[2][q];
        }
    }
}

template <typename TA, typename TB>
__global__ void __launch_bounds__(kRedThreads)
reduce_pass1(int64_t count, const TA *__restrict__ a, const TB *__restrict__ b, double *__restrict__ part) {
    double m0 = 0.0, m1 = 0.0, s = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count; q += stride) {
        const double x = (double)a[q], y = (double)b[q];
        m0 = nan_max(m0, fabs(x - y));
        m1 = nan_max(m1, fabs(y));
        s = __fma_rn(x, y, s);
    }
    block_reduce3(m0, m1, s);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x + 0] = m0;
        part[3 * blockIdx.x + 1] = m1;
        part[3 * blockIdx.x + 2] = s;
    }
}

__global__ void __launch_bounds__(kRedThreads)
reduce_pass2(int nparts, const double *__restrict__ part, double *__restrict__ out) {
    double m0 = 0.0, m1 = 0.0, s = 0.0;
    for (int q = threadIdx.x; q < nparts; q += blockDim.x) {
        m0 = nan_max(m0, part[3 * q + 0]);
        m1 = nan_max(m1, part[3 * q + 1]);
        s += part[3 * q + 2];
    }
    block_reduce3(m0, m1, s);
    if (threadIdx.x == 0) { out[0] = m0; out[1] = m1; out[2] = s; }
}

template <typename TA, typename TB>
static int launch_reduce(int64_t count, const void *a, const void *b, double *out, double *part,
                         int blocks, cudaStream_t s) {
    reduce_pass1<TA, TB><<<blocks, kRedThreads, 0, s>>>(count, (const TA *)a, (const TB *)b, part);
    int st = launch_status();
    if (st != SEMAX_OK) return st;
    reduce_pass2<<<1, kRedThreads, 0, s>>>(blocks, part, out);
    return launch_status();
}

}  // namespace semax

using namespace semax;

extern "C" int semax_reduce_workspace_size(int64_t count, size_t *bytes) {
    if (count < 0 || !bytes) return SEMAX_EINVAL;
    *bytes = (size_t)reduce_blocks(count) * 3 * sizeof(double);
    return SEMAX_OK;
}

extern "C" int semax_reduce(int64_t count, const void *a, int a_prec, const void *b, int b_prec,
                            double *out, void *workspace, size_t ws_bytes, void *stream) {
    if (count < 0 || !out) return SEMAX_EINVAL;
    if ((a_prec != SEMAX_F64 && a_prec != SEMAX_F32) || (b_prec != SEMAX_F64 && b_prec != SEMAX_F32))
        return SEMAX_EINVAL;
    if (count > 0 && (!a || !b)) return SEMAX_EINVAL;
    if (((uintptr_t)out & 7u) || ((uintptr_t)workspace & 7u)) return SEMAX_EALIGN;
    const int blocks = reduce_blocks(count);
    if (!workspace || ws_bytes < (size_t)blocks * 3 * sizeof(double)) return SEMAX_EWORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    double *part = (double *)workspace;
    if (a_prec == SEMAX_F64 && b_prec == SEMAX_F64) return launch_reduce<double, double>(count, a, b, out, part, blocks, s);
    if (a_prec == SEMAX_F32 && b_prec == SEMAX_F64) return launch_reduce<float, double>(count, a, b, out, part, blocks, s);
    if (a_prec == SEMAX_F64 && b_prec == SEMAX_F32) return launch_reduce<double, float>(count, a, b, out, part, blocks, s);
    return launch_reduce<float, float>(count, a, b, out, part, blocks, s);
}

// ---------------------------------------------------------------- no-allocation form
//
// Some callers cannot call cudaMalloc: a legacy Fortran or C solver that hands
// the library only its own arrays (and owns every device allocation itself),
// code running where the allocator must not be touched (inside a memory pool
// owned by another runtime, a real-time loop that forbids allocation), or a
// caller that has no spare buffer to lend.  semax_reduce_noalloc gives them the
// same FP64 reduction without a workspace argument: its per-block partials live
// in the file-scope array below, which every GPU that loads the library holds
// until the process exits.

namespace semax {

// Partials of the fixed partition: at most kRedMaxBlocks blocks x 3 doubles
// (24 KiB per device).
constexpr int kNoAllocBlocks = kRedMaxBlocks;
static __device__ __align__(256) double g_reduce_scratch[3 * kNoAllocBlocks];

constexpr int kMaxDevices = 64;

// The cached device address of g_reduce_scratch, per device ordinal, with the
// id of the context it was looked up in: after a device reset the runtime
// makes a new primary context, where the array lives at an address that must
// be looked up again.
struct ScratchCache {
    unsigned long long ctx_id = 0;
    double *ptr = nullptr;
};
static ScratchCache g_scratch[kMaxDevices];
static std::mutex g_scratch_mutex;

// Unique id of the calling thread's current context (0 if none, or if the
// driver entry points are unavailable), through the runtime's driver entry
// point query, so that the library does not link the driver library itself.
static unsigned long long current_context_id() {
    using GetCurrent = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Device address of g_reduce_scratch in the current device's context.  In
// host code the symbol names a host-side stand-in, so the address must come
// from cudaGetSymbolAddress with that device current; it is looked up on the
// first call in each context and cached.
static int noalloc_scratch(double **out) {
    int dev = 0;
    int st = cuda_status(cudaGetDevice(&dev));
    if (st != SEMAX_OK) return st;
    if (dev < 0 || dev >= kMaxDevices) return SEMAX_EINVAL;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    const unsigned long long id = current_context_id();
    ScratchCache &c = g_scratch[dev];
    if (!c.ptr || id == 0 || c.ctx_id != id) {
        void *addr = nullptr;
        st = cuda_status(cudaGetSymbolAddress(&addr, g_reduce_scratch));
        if (st != SEMAX_OK) return st;
        c.ptr = static_cast<double *>(addr);
        c.ctx_id = current_context_id();   // the lookup made the context current if it was not
    }
    *out = c.ptr;
    return SEMAX_OK;
}

}  // namespace semax

extern "C" int semax_reduce_noalloc(int64_t count, const void *a, int a_prec, const void *b, int b_prec,
                                    double *out, void *stream) {
    if (count < 0 || !out) return SEMAX_EINVAL;
    if ((a_prec != SEMAX_F64 && a_prec != SEMAX_F32) || (b_prec != SEMAX_F64 && b_prec != SEMAX_F32))
        return SEMAX_EINVAL;
    if (count > 0 && (!a || !b)) return SEMAX_EINVAL;
    if ((uintptr_t)out & 7u) return SEMAX_EALIGN;
    const int blocks = reduce_blocks(count);
    if (blocks > kNoAllocBlocks) return SEMAX_EWORKSPACE;   // partials would not fit the static scratch
    double *part = nullptr;
    int st = noalloc_scratch(&part);
    if (st != SEMAX_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (a_prec == SEMAX_F64 && b_prec == SEMAX_F64) return launch_reduce<double, double>(count, a, b, out, part, blocks, s);
    if (a_prec == SEMAX_F32 && b_prec == SEMAX_F64) return launch_reduce<float, double>(count, a, b, out, part, blocks, s);
    if (a_prec == SEMAX_F64 && b_prec == SEMAX_F32) return launch_reduce<double, float>(count, a, b, out, part, blocks, s);
    return launch_reduce<float, float>(count, a, b, out, part, blocks, s);
}
