// Arithmetic-pipe probe for the roofline of the plain kernels: every thread
// runs independent chains of dependent fused multiply-adds (FP64 or FP32)
// for `iters` steps and writes one sum, so the measured rate is the FMA
// pipe's sustained throughput with latency hidden by the chains and warps.
// Not part of the operator.
#include "common.cuh"

namespace semax {

// Chains per thread: four in FP64, each with its own multiplier and addend
// registers (eight chains, or operands shared by all chains, ran 10-15 %
// slower on GB300); eight in FP32 sharing one multiplier and addend (own
// operands per chain ran a third slower there).
template <typename T>
__host__ __device__ constexpr int probe_chains() { return sizeof(T) == 8 ? 4 : 8; }

template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(int iters, T b, T c, T *__restrict__ sink) {
    constexpr int CH = probe_chains<T>();
    constexpr bool kOwn = sizeof(T) == 8;   // per-chain operand registers
    T a[CH], bq[CH], cq[CH];
#pragma unroll
    for (int q = 0; q < CH; ++q) {
        a[q] = (T)(threadIdx.x + q) * c;
        bq[q] = kOwn ? b - (T)q * (T)1e-6 * (T)(1 - b) : b;   // each < 1
        cq[q] = kOwn ? c * (T)(q + 1) : c;
    }
    for (int it = 0; it < iters; it += 4) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int q = 0; q < CH; ++q) a[q] = fma(a[q], bq[q], cq[q]);
    }
    T s = 0;
#pragma unroll
    for (int q = 0; q < CH; ++q) s += a[q];
    sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace semax

using namespace semax;

extern "C" int semax_fma_probe(int prec, int blocks, int iters, void *sink, double *flops, void *stream) {
    if ((prec != SEMAX_F64 && prec != SEMAX_F32) || blocks <= 0 || iters <= 0 || (iters & 3) || !sink || !flops)
        return SEMAX_EINVAL;
    if (((uintptr_t)sink % (prec == SEMAX_F64 ? 8u : 4u)) != 0) return SEMAX_EALIGN;
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == SEMAX_F64)
        fma_probe_kernel<double><<<blocks, 256, 0, s>>>(iters, 0.9999999999, 1e-9, (double *)sink);
    else
        fma_probe_kernel<float><<<blocks, 256, 0, s>>>(iters, 0.9999999f, 1e-7f, (float *)sink);
    const int chains = prec == SEMAX_F64 ? probe_chains<double>() : probe_chains<float>();
    *flops = 2.0 * chains * (double)iters * 256.0 * (double)blocks;
    return launch_status();
}
