// FP32 instantiation of the plain Ax kernels.
#include "ax_plain.cuh"

namespace semax {
template int launch_plain<float, false>(int64_t, int, const TileConfig &, const float *, const float *,
                                         const float *, float *, const float *, Helm<float>, cudaStream_t);
}  // namespace semax
