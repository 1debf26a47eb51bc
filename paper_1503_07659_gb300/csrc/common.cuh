// Shared host/device helpers of libsemax: status plumbing, argument checks,
// cache-hinted global loads.  No operator arithmetic lives here.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "semax.h"

namespace semax {

constexpr int kMaxN = 15;          // n = N + 1 <= 16
constexpr int kNumSMsHint = 152;   // GB300; the runtime value is queried

// last CUDA error seen by a libsemax call on this host thread
int &last_cuda_error();

inline int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return SEMAX_OK;
    last_cuda_error() = (int)e;
    return SEMAX_ECUDA;
}

// Status of the launch just made (clears the sticky-free launch error state).
inline int launch_status() { return cuda_status(cudaGetLastError()); }

inline bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

inline bool overlaps(const void *a, size_t abytes, const void *b, size_t bbytes) {
    const uintptr_t a0 = (uintptr_t)a, a1 = a0 + abytes;
    const uintptr_t b0 = (uintptr_t)b, b1 = b0 + bbytes;
    return abytes && bbytes && a0 < b1 && b0 < a1;
}

// Common validation of (E, N, u, G, D, w).  Returns SEMAX_OK or an error.
template <typename T>
inline int check_args(int64_t E, int N, const T *u, const T *G, const T *D, const T *w) {
    if (E < 0) return SEMAX_EINVAL;
    if (N < 1 || N > kMaxN) return SEMAX_EUNSUPPORTED_N;
    if (E == 0) return SEMAX_OK;
    if (!u || !G || !D || !w) return SEMAX_EINVAL;
    if (!aligned16(u) || !aligned16(G) || !aligned16(w)) return SEMAX_EALIGN;
    if (((uintptr_t)D % alignof(T)) != 0) return SEMAX_EALIGN;
    const size_t n = (size_t)N + 1, n3 = n * n * n;
    const size_t ub = (size_t)E * n3 * sizeof(T);
    if (overlaps(w, ub, u, ub) || overlaps(w, ub, G, 6 * ub) || overlaps(w, ub, D, n * n * sizeof(T)))
        return SEMAX_EALIAS;
    return SEMAX_OK;
}

int device_sm_count();

// Polls a staging wait of the tensor-core kernels makes before it gives up;
// the limit of each element's first wait is read at launch from a
// process-wide setting (semax_set_wait_polls), the drain wait after a
// timeout always takes the default.
constexpr int kDefaultWaitPolls = 1 << 20;
int first_wait_polls();

// ---------------------------------------------------------------- device side

// Streaming read-once loads: do not keep the line in L1.
__device__ __forceinline__ double ld_stream(const double *p) {
    double v;
    asm volatile("ld.global.nc.L1::no_allocate.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ float ld_stream(const float *p) {
    float v;
    asm volatile("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ float4 ld_stream4(const float4 *p) {
    float4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
    return v;
}

// Copy `count` values global -> shared, 16-byte vectors when both ends allow.
template <typename T>
__device__ __forceinline__ void copy_to_smem(T *dst, const T *__restrict__ src, int count) {
    const bool vec = ((((uintptr_t)src) | ((uintptr_t)dst)) & 15u) == 0 &&
                     ((count * (int)sizeof(T)) & 15) == 0;
    if (vec) {
        const int nv = count * (int)sizeof(T) / 16;
        const float4 *s4 = reinterpret_cast<const float4 *>(src);
        float4 *d4 = reinterpret_cast<float4 *>(dst);
        for (int q = threadIdx.x; q < nv; q += blockDim.x) d4[q] = ld_stream4(s4 + q);
    } else {
        for (int q = threadIdx.x; q < count; q += blockDim.x) dst[q] = ld_stream(src + q);
    }
}

}  // namespace semax
