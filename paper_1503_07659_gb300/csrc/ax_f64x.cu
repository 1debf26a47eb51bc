// Launcher and C ABI of the double-float FP64-accurate Ax (ax_f64x.cuh).
#include "ax_f64x.cuh"

namespace semax {
namespace dfx {

template <int n>
static int launch(int64_t E, const double *u, const double *G, const double *D, double *w, cudaStream_t s) {
    constexpr int epb = elems_per_tile<n>();
    const size_t smem = smem_bytes<n>(epb);
    auto kern = ax_f64x_kernel<n>;
    int st = cuda_status(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (st != SEMAX_OK) return st;
    st = cuda_status(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                          (int)cudaSharedmemCarveoutMaxShared));
    if (st != SEMAX_OK) return st;
    const int64_t tiles = (E + epb - 1) / epb;
    if (tiles > 0x7fffffffLL) return SEMAX_EINVAL;
    kern<<<(unsigned)tiles, kThreads, smem, s>>>(E, u, G, D, w);
    return launch_status();
}

}  // namespace dfx
}  // namespace semax

using namespace semax;

extern "C" int sem_ax_f64x(int64_t E, int N, const double *u, const double *G, const double *D, double *w,
                           void *stream) {
    int st = check_args(E, N, u, G, D, w);
    if (st != SEMAX_OK || E == 0) return st;
    cudaStream_t s = (cudaStream_t)stream;
    switch (N + 1) {
        case 2: return dfx::launch<2>(E, u, G, D, w, s);
        case 4: return dfx::launch<4>(E, u, G, D, w, s);
        case 6: return dfx::launch<6>(E, u, G, D, w, s);
        case 8: return dfx::launch<8>(E, u, G, D, w, s);
        case 10: return dfx::launch<10>(E, u, G, D, w, s);
        case 12: return dfx::launch<12>(E, u, G, D, w, s);
        case 14: return dfx::launch<14>(E, u, G, D, w, s);
        case 16: return dfx::launch<16>(E, u, G, D, w, s);
        default: return sem_ax(E, N, u, G, D, w, stream);   // odd n: the FP64 tile
    }
}
