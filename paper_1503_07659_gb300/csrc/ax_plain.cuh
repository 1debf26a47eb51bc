// Plain (one order per launch) Ax kernels, FP64 and FP32 CUDA-core forms.
#pragma once

#include "ax_tile.cuh"

namespace semax {

struct TileConfig {
    int epb;   // elements per CTA tile
    int map;   // MAP_NODE or MAP_COLUMN
    int threads;
};

// Default tile shapes, from a sweep of (mapping, elements per tile, block
// size) on GB300: even n takes the even/odd line mapping (the GLL derivative
// is centro-antisymmetric), FP64 with 256 threads and 256/n^2 elements per
// tile, FP32 up to n = 8 with small 64-thread tiles (many resident CTAs hide
// the load latency best) and one element per 256-thread tile above; odd n
// takes one (i,j) column per thread.
template <typename T>
inline TileConfig default_tile(int n) {
    TileConfig c;
    if (n % 2 == 0) {
        c.map = MAP_EO;
        const int threads = (sizeof(T) == 4 && n <= 8) ? 64 : 256;
        c.threads = threads;
        c.epb = threads / (n * n) > 0 ? threads / (n * n) : 1;
    } else {
        c.map = MAP_COLUMN;
        c.epb = 256 / (n * n) > 0 ? 256 / (n * n) : 1;
        c.threads = round_up(c.epb * n * n, 32);
    }
    return c;
}

// Registers are capped for three resident CTAs per SM wherever three tiles
// fit in shared memory: FP64 up to n = 8, FP32 at n > 12.  FP32 up to n = 12
// takes 64 registers (four CTAs of 256 threads, or more of 64), measured 6-8 %
// faster than 80; at n = 16 three CTAs with 80 registers are faster.
template <typename T, int n, int MAP, bool HELM>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 ? (n <= 12 ? 4 : 3) : (n <= 8 ? 3 : 1)))
ax_plain_kernel(int64_t E, int epb, const T *__restrict__ u, const T *__restrict__ G,
                const T *__restrict__ D, T *__restrict__ w, const T *__restrict__ scale, Helm<T> helm) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int n3 = n * n * n;
    T *sD = reinterpret_cast<T *>(smem_raw);
    T *buf = sD + d_slots<T>(n);
    const int64_t e0 = (int64_t)blockIdx.x * epb;
    const int cnt = (int)(E - e0 < epb ? E - e0 : epb);
    if constexpr (sizeof(T) == 4) {
        // FP32: the tile's G into L2 first, so that the column pass's loads of
        // it wait on L2 rather than on HBM
        const char *src = reinterpret_cast<const char *>(G + e0 * 6 * n3);
        const int lines = (int)(((size_t)cnt * 6 * n3 * sizeof(T)) / 128);
#pragma unroll 1
        for (int q = threadIdx.x; q < lines; q += blockDim.x)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(src + 128 * (size_t)q));
    }
    load_D<T, n>(D, sD);
    if constexpr (HELM) helm.B += e0 * n3;
    ax_tile<T, n, MAP, HELM>(cnt, u + e0 * n3, G + e0 * 6 * n3, w + e0 * n3,
                             scale ? scale + e0 : nullptr, helm, sD, buf);
}

template <typename T, bool HELM, int n, int MAP>
int launch_plain_nm(int64_t E, const TileConfig &c, const T *u, const T *G, const T *D, T *w,
                    const T *scale, Helm<T> helm, cudaStream_t s) {
    auto kern = ax_plain_kernel<T, n, MAP, HELM>;
    const size_t smem = tile_smem_bytes<T>(n, c.epb, MAP);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_status(e);
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return cuda_status(e);
    }
    const int64_t tiles = (E + c.epb - 1) / c.epb;
    if (tiles > 0x7fffffffLL) return SEMAX_EINVAL;
    kern<<<(unsigned)tiles, c.threads, smem, s>>>(E, c.epb, u, G, D, w, scale, helm);
    return launch_status();
}

template <typename T, bool HELM, int n>
int launch_plain_n(int64_t E, const TileConfig &c, const T *u, const T *G, const T *D, T *w,
                   const T *scale, Helm<T> helm, cudaStream_t s) {
    if (c.epb < 1 || c.threads < 32 || c.threads > 256 || (c.threads & 31)) return SEMAX_EINVAL;
    if (c.map == MAP_COLUMN) {
        if (c.epb * n * n > c.threads) return SEMAX_EINVAL;
        return launch_plain_nm<T, HELM, n, MAP_COLUMN>(E, c, u, G, D, w, scale, helm, s);
    }
    if (c.map == MAP_EO && n % 2 == 0)
        return launch_plain_nm<T, HELM, n, MAP_EO>(E, c, u, G, D, w, scale, helm, s);
    return launch_plain_nm<T, HELM, n, MAP_NODE>(E, c, u, G, D, w, scale, helm, s);
}

// Launch the plain kernel for order N with tile shape c.  HELM selects the
// Helmholtz form (helm.B, h1, h2); otherwise helm is ignored.
template <typename T, bool HELM = false>
int launch_plain(int64_t E, int N, const TileConfig &c, const T *u, const T *G, const T *D, T *w,
                 const T *scale, Helm<T> helm, cudaStream_t s) {
    switch (N + 1) {
#define SEMAX_CASE(nn) \
    case nn: return launch_plain_n<T, HELM, nn>(E, c, u, G, D, w, scale, helm, s);
        SEMAX_CASE(2) SEMAX_CASE(3) SEMAX_CASE(4) SEMAX_CASE(5) SEMAX_CASE(6) SEMAX_CASE(7)
        SEMAX_CASE(8) SEMAX_CASE(9) SEMAX_CASE(10) SEMAX_CASE(11) SEMAX_CASE(12) SEMAX_CASE(13)
        SEMAX_CASE(14) SEMAX_CASE(15) SEMAX_CASE(16)
#undef SEMAX_CASE
        default: return SEMAX_EUNSUPPORTED_N;
    }
}

// Explicit instantiations live in ax_f64.cu, ax_f32.cu and ax_helm.cu.
extern template int launch_plain<double, false>(int64_t, int, const TileConfig &, const double *,
                                                const double *, const double *, double *,
                                                const double *, Helm<double>, cudaStream_t);
extern template int launch_plain<float, false>(int64_t, int, const TileConfig &, const float *,
                                               const float *, const float *, float *, const float *,
                                               Helm<float>, cudaStream_t);
extern template int launch_plain<double, true>(int64_t, int, const TileConfig &, const double *,
                                               const double *, const double *, double *,
                                               const double *, Helm<double>, cudaStream_t);

}  // namespace semax
