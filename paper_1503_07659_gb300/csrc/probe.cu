// Arithmetic-pipe probe for the roofline of the plain kernels: every thread
// runs CH independent chains of dependent fused multiply-adds (FP64 or FP32)
// for `iters` steps and writes one sum, so the measured rate is the FMA
// pipe's sustained throughput with latency hidden by the chains and warps.
// Not part of the operator.
#include "common.cuh"

namespace semax {

constexpr int kProbeChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(int iters, T b, T c, T *__restrict__ sink) {
    T a[kProbeChains];
#pragma unroll
    for (int q = 0; q < kProbeChains; ++q) a[q] = (T)(threadIdx.x + q) * c;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < kProbeChains; ++q) a[q] = fma(a[q], b, c);
    }
    T s = 0;
#pragma unroll
    for (int q = 0; q < kProbeChains; ++q) s += a[q];
    sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace semax

using namespace semax;

extern "C" int semax_fma_probe(int prec, int blocks, int iters, void *sink, double *flops, void *stream) {
    if ((prec != SEMAX_F64 && prec != SEMAX_F32) || blocks <= 0 || iters <= 0 || !sink || !flops)
        return SEMAX_EINVAL;
    if (((uintptr_t)sink % (prec == SEMAX_F64 ? 8u : 4u)) != 0) return SEMAX_EALIGN;
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == SEMAX_F64)
        fma_probe_kernel<double><<<blocks, 256, 0, s>>>(iters, 0.9999999999, 1e-9, (double *)sink);
    else
        fma_probe_kernel<float><<<blocks, 256, 0, s>>>(iters, 0.9999999f, 1e-7f, (float *)sink);
    *flops = 2.0 * kProbeChains * (double)iters * 256.0 * (double)blocks;
    return launch_status();
}
